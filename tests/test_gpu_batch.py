"""GPU parity of the generic batched path on host-submitted irregular tasks
(Section 3.1 combining, Section 3.2 chare table and sorted pack):
uneven task sizes, long lists (merged sort path), eviction under a small
pool, staging-budget waves, error paths, determinism and edge cases."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import EPS2, TOL, make_pool, per_task_errors, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    return gcharm


def uneven(n_ids=20000, n_tasks=200, seed=3, t_range=(1, 100), s_range=(1, 9000)):
    x = inputs.merger(3 * n_ids // 4, n_ids // 4, seed)
    to, tg, so, sr = inputs.uneven_tasks(n_ids, n_tasks, seed + 1, t_range, s_range)
    return x, to, tg, so, sr


def submit_gravity(pool, to, tg, so, sr, task_ids=None):
    return pool.submit_csr(np.zeros(len(to) - 1, np.uint32), to, tg, so, sr, task_ids=task_ids)


def test_uneven_tasks_vs_oracle(gc, orc):
    x, to, tg, so, sr = uneven()
    n = x.shape[0]
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    b = submit_gravity(pool, to, tg, so, sr)
    pool.flush()
    pool.wait(b)
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    got = pool.values()
    errs = per_task_errors(got, ref, to)
    assert errs.max() <= TOL, errs.max()
    # totals: ids repeat across tasks; FP64 sums in admission order
    tot_ref = orc.reduce(tg, ref, n)
    u = np.unique(tg)
    assert rel_l2(pool.totals(u)[:, :3], tot_ref[u, :3]) <= TOL
    # chare table and pack permutation
    R = orc.Residency(n, n)
    rc, r = R.flush(np.concatenate([tg, sr]), 1)
    st, ss = pool.entry_slots()
    assert np.array_equal(np.concatenate([st, ss]), r["slots"])
    pt, ps = pool.pack_perm()
    assert np.array_equal(pt, orc.pack_perm_batch(to, st))
    assert np.array_equal(ps, orc.pack_perm_batch(so, ss))
    s = pool.stats()
    assert s["last_unique"] == r["unique"]
    assert sum(s["reuse_hist"]) == r["unique"]
    assert s["reuse_hist"][0] == int((r["reuse"] == 1).sum())
    assert s["reuse_hist"][7] == int((r["reuse"] > 64).sum())
    pool.close()


def test_results_by_task_id(gc, orc):
    x, to, tg, so, sr = uneven(n_tasks=20)
    n = x.shape[0]
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    tids = np.arange(1000, 1020, dtype=np.uint64)
    submit_gravity(pool, to, tg, so, sr, task_ids=tids)
    pool.flush()
    pick = [1013, 1002]
    rows = int((to[14] - to[13]) + (to[3] - to[2]))
    got = gc.value(pool.read_results(np.array(pick, np.uint64), rows))
    all_rows = pool.values()
    exp = np.concatenate([all_rows[to[13]:to[14]], all_rows[to[2]:to[3]]])
    assert np.array_equal(got, exp)
    pool.close()


def test_eviction_sequence_matches_oracle(gc, orc):
    n, cap = 3000, 700
    x = inputs.plummer(n, 8)
    pool = make_pool(gc, torch, n, cap)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    R = orc.Residency(n, cap)
    g = inputs.rng(12)
    for epoch in range(1, 9):
        k = 6
        nt = g.integers(1, 20, k)
        ns = g.integers(1, 60, k)
        to = np.concatenate([[0], np.cumsum(nt)]).astype(np.uint64)
        so = np.concatenate([[0], np.cumsum(ns)]).astype(np.uint64)
        hot = g.integers(0, 400, int(to[-1] + so[-1]))
        cold = g.integers(0, n, int(to[-1] + so[-1]))
        ids = np.where(g.random(len(hot)) < 0.5, hot, cold).astype(np.uint32)
        tg, sr = ids[:to[-1]], ids[to[-1]:]
        submit_gravity(pool, to, tg, so, sr)
        pool.flush()
        rc, r = R.flush(np.concatenate([tg, sr]), epoch)
        assert rc == 0
        s2o, o2s, lu = pool.residency()
        assert np.array_equal(s2o, R.slot_of_id), epoch
        assert np.array_equal(o2s, R.id_of_slot), epoch
        assert np.array_equal(pool.evicted(), r["evicted"]), epoch
        ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
        errs = per_task_errors(pool.values(), ref, to)
        assert errs.max() <= TOL
    assert pool.stats()["evictions"] > 0
    pool.close()


def test_pool_full_is_reported_and_pool_stays_usable(gc):
    n = 500
    x = inputs.plummer(n, 9)
    pool = make_pool(gc, torch, n, 50)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    to = np.array([0, 10], np.uint64)
    so = np.array([0, 100], np.uint64)
    submit_gravity(pool, to, np.arange(10, dtype=np.uint32), so, np.arange(100, 200, dtype=np.uint32))
    with pytest.raises(gc.GcError) as e:
        pool.flush()
    assert e.value.code == gc.GC_ERR_POOL_FULL
    so = np.array([0, 30], np.uint64)
    submit_gravity(pool, to, np.arange(10, dtype=np.uint32), so, np.arange(100, 130, dtype=np.uint32))
    pool.flush()
    pool.close()


def test_unknown_id_and_bad_tasks(gc):
    n = 100
    x = inputs.plummer(n, 10)
    pool = make_pool(gc, torch, 2 * n, 2 * n, staging_budget_bytes=16 * 64)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    to = np.array([0, 2], np.uint64)
    so = np.array([0, 3], np.uint64)
    submit_gravity(pool, to, np.array([1, 2], np.uint32), so, np.array([3, 150, 4], np.uint32))
    with pytest.raises(gc.GcError) as e:
        pool.flush()
    assert e.value.code == gc.GC_ERR_UNKNOWN_ID
    with pytest.raises(gc.GcError) as e:   # id >= id_capacity rejected on the host
        pool.upload(np.array([5000], np.uint32), x[:1])
    assert e.value.code == gc.GC_ERR_ARG
    with pytest.raises(gc.GcError) as e:   # self task with sources
        pool.submit_csr(np.array([2], np.uint32), to, np.array([1, 2], np.uint32), so,
                        np.array([3, 4, 5], np.uint32))
    assert e.value.code == gc.GC_ERR_ARG
    with pytest.raises(gc.GcError) as e:   # one task larger than the staging budget
        submit_gravity(pool, to, np.array([1, 2], np.uint32), np.array([0, 80], np.uint64),
                       np.arange(80, dtype=np.uint32))
    assert e.value.code == gc.GC_ERR_BUDGET
    # still usable
    submit_gravity(pool, to, np.array([1, 2], np.uint32), so, np.array([3, 4, 5], np.uint32))
    pool.flush()
    assert pool.result_rows() == 2
    pool.close()


def test_waves_equal_single_launch(gc):
    x, to, tg, so, sr = uneven(n_tasks=120, s_range=(1, 3000))
    n = x.shape[0]
    outs = []
    for budget in [0, 16 * 20000]:
        pool = make_pool(gc, torch, n, n, staging_budget_bytes=budget)
        pool.upload(np.arange(n, dtype=np.uint32), x)
        submit_gravity(pool, to, tg, so, sr)
        pool.flush()
        outs.append((pool.results(), pool.totals(np.arange(n, dtype=np.uint32)),
                     pool.stats()["last_waves"]))
        pool.close()
    assert outs[0][2] == 1 and outs[1][2] > 1
    # waves allocate slots wave by wave, so the pack order (and the FP32
    # summation order) may differ: equal within the force tolerance
    ref = gc.value(outs[0][0])
    errs = per_task_errors(gc.value(outs[1][0]), ref, to)
    assert errs.max() <= TOL
    assert rel_l2(outs[1][1][:, :3], outs[0][1][:, :3]) <= TOL


def test_deterministic_repeat(gc):
    x, to, tg, so, sr = uneven(n_tasks=80)
    n = x.shape[0]
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    res = []
    for _ in range(2):
        pool.reset_totals()
        submit_gravity(pool, to, tg, so, sr)
        pool.flush()
        res.append((pool.results(), pool.totals(np.arange(n, dtype=np.uint32))))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert pool.stats()["last_hits"] == pool.stats()["last_unique"]   # second pass: all reused
    pool.close()


def test_edge_cases(gc, orc):
    n = 64
    x = inputs.plummer(n, 11)
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    pool.flush()                                  # empty batch: no-op
    # task with no sources, task with no targets, duplicate source ids, a
    # single target with a single (self) source
    to = np.array([0, 3, 3, 4, 5], np.uint64)
    so = np.array([0, 0, 5, 9, 10], np.uint64)
    tg = np.array([1, 2, 3, 7, 9], np.uint32)
    sr = np.array([4, 5, 6, 7, 8, 11, 11, 11, 12, 9], np.uint32)
    pool.submit_tasks([dict(task_id=0, kind=0, targets=tg[0:3], sources=[]),
                       dict(task_id=1, kind=0, targets=[], sources=sr[0:5]),
                       dict(task_id=2, kind=0, targets=tg[3:4], sources=sr[5:9]),
                       dict(task_id=3, kind=0, targets=tg[4:5], sources=sr[9:10])])
    pool.flush()
    got = pool.values()
    assert got.shape[0] == 5
    assert np.all(got[:3] == 0)
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    assert rel_l2(got[3:4, :3], ref[3:4, :3]) <= TOL
    assert np.all(got[4, :3] == 0)               # self term: dx = 0
    assert got[4, 3] == pytest.approx(ref[4, 3], rel=1e-6)
    pool.close()


def test_wait_expiry_reported_and_pool_stays_usable(gc, orc):
    """The bounded barrier wait of the interaction kernels gives up instead of
    hanging: its expiry path (a wait on a barrier nothing arrives at) sets
    the timeout status, the next wait reports GC_ERR_TIMEOUT once, and the
    same pool then runs batches that match the oracle."""
    x, to, tg, so, sr = uneven(n_ids=4000, n_tasks=30, seed=41, s_range=(1, 500))
    n = x.shape[0]
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    b0 = submit_gravity(pool, to, tg, so, sr)
    pool.flush()
    pool.wait(b0)
    pool.check_wait_expiry(2048)
    b1 = submit_gravity(pool, to, tg, so, sr)
    pool.flush()
    with pytest.raises(gc.GcError) as e:
        pool.wait(b1)
    assert e.value.code == gc.GC_ERR_TIMEOUT
    pool.wait(b1)                       # the status was cleared by the report
    assert per_task_errors(pool.values(), ref, to).max() <= TOL
    b2 = submit_gravity(pool, to, tg, so, sr)
    pool.flush()
    pool.wait(b2)
    assert per_task_errors(pool.values(), ref, to).max() <= TOL
    for bad in (0, (1 << 24) + 1):
        with pytest.raises(gc.GcError) as e:
            pool.check_wait_expiry(bad)
        assert e.value.code == gc.GC_ERR_ARG
    pool.close()


def test_reset_totals_semantics(gc):
    """A reset zeroes the per-id totals for every later reader: a read right
    after it sees zeros, the next batch's totals hold that batch alone, and
    batches flushed back to back without a reset accumulate."""
    x, to, tg, so, sr = uneven(n_ids=3000, n_tasks=20, seed=51, s_range=(1, 300))
    n = x.shape[0]
    ids = np.arange(n, dtype=np.uint32)
    pool = make_pool(gc, torch, n, n)
    pool.upload(ids, x)
    b = submit_gravity(pool, to, tg, so, sr)
    pool.flush()
    pool.wait(b)
    one = pool.totals(ids)
    assert np.abs(one).sum() > 0
    pool.reset_totals()
    assert not pool.totals(ids).any()
    pool.reset_totals()
    for _ in range(2):                  # two batches in flight, one reset before them
        b = submit_gravity(pool, to, tg, so, sr)
        pool.flush()
    pool.wait(b)
    np.testing.assert_allclose(pool.totals(ids), 2 * one, rtol=1e-12, atol=1e-300)
    pool.reset_totals()
    b = submit_gravity(pool, to, tg, so, sr)
    pool.flush()
    pool.wait(b)
    assert np.array_equal(pool.totals(ids), one)
    pool.close()


def test_per_id_totals_exact_small_and_large_batches(gc, orc):
    """The per-id totals are the rows' FP64 values s - c summed per id in
    admission order.  Batches of at most 2048 rows take a one-block path,
    larger ones sort (id, row) first; both must give the oracle's reduction
    of the same row values bit for bit, and so must a graph replay of a
    small batch."""
    n = 600                                   # few ids: they repeat across tasks
    x = inputs.plummer(n, inputs.SEED_BASE + 21)
    for n_tasks, t_range in [(40, (1, 60)), (300, (1, 40))]:
        to, tg, so, sr = inputs.uneven_tasks(n, n_tasks, inputs.SEED_BASE + 22, t_range,
                                             (1, 400))
        rows = int(to[-1])
        assert (rows <= 2048) == (n_tasks == 40)
        pool = make_pool(gc, torch, n, n)
        pool.upload(np.arange(n, dtype=np.uint32), x)
        b = submit_gravity(pool, to, tg, so, sr)
        pool.flush()
        pool.wait(b)
        vals = pool.values()                  # (rows, 4) FP64 s - c
        ref = orc.reduce(tg, vals, n)
        u = np.unique(tg)
        got = pool.totals(u)
        assert np.array_equal(got, ref[u]), n_tasks
        pool.close()
        if n_tasks == 40:   # the same batch captured: the capture run and a replay
            pool = make_pool(gc, torch, n, n)
            pool.upload(np.arange(n, dtype=np.uint32), x)
            submit_gravity(pool, to, tg, so, sr)
            g = gc.Graph(pool)
            gref = orc.reduce(tg, gc.value(g.results()), n)
            assert np.array_equal(pool.totals(u), gref[u])
            pool.reset_totals()
            g.launch()
            g.wait()
            assert np.array_equal(pool.totals(u), gref[u])
            g.close()
            pool.close()


def test_async_upload_and_totals_read_match_sync(gc):
    """Uploads and totals reads queued in stream order (the host waits once,
    at the end) give the same per-id totals, step by step, as the
    synchronous calls."""
    n = 6000
    ids = np.arange(n, dtype=np.uint32)
    xs = [inputs.plummer(n, inputs.SEED_BASE + 31)]
    for k in range(2):
        xs.append(inputs.drift(xs[-1], inputs.SEED_BASE + 32 + k))
    ps = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
    pa = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
    sync_tot = []
    for x in xs:
        ps.upload(ids, x)
        ps.reset_totals()
        ps.build_nbody_resident(n, 32, 7, 10)
        ps.flush()
        sync_tot.append(ps.totals(ids))
    outs = [np.zeros((n, 4), np.float64) for _ in xs]
    hx = [np.ascontiguousarray(x, np.float32) for x in xs]
    for k, x in enumerate(hx):
        pa.upload_async(ids, x)
        pa.reset_totals()
        pa.build_nbody_resident(n, 32, 7, 10)
        pa.flush()
        pa.totals_async(ids, outs[k])
    pa.join(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for k in range(len(xs)):
        assert np.array_equal(outs[k], sync_tot[k]), k
    # an id beyond the capacity is skipped on the device; the next flush says so
    bad = ids.copy()
    bad[7] = 10 * n
    pa.upload_async(bad, hx[0])
    pa.build_nbody_resident(n, 32, 7, 10)
    with pytest.raises(gc.GcError) as e:
        pa.flush()
    assert e.value.code == gc.GC_ERR_UNKNOWN_ID
    torch.cuda.synchronize()
    with pytest.raises(ValueError):
        pa.upload_async(ids.astype(np.int64), hx[0])
    with pytest.raises(ValueError):
        pa.totals_async(ids, np.zeros((n, 4), np.float32))
    ps.close()
    pa.close()
