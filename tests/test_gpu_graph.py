"""GPU tests of the replayable graph form of a combined batch: the capture
run and every replay match the FP64 oracle; a replay repeats the capture
run's rows bit for bit; replays read values re-uploaded in place; per-id
totals accumulate once per replay; a replay after the chare table changed
is refused; multi-wave batches and LJ batches replay as well."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import EPS2, RC2, RC2_GRID, TOL, make_pool, per_task_errors, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    return gcharm


def uneven(n=12000, tasks=150, seed=31, s_range=(1, 3000)):
    x = inputs.merger(3 * n // 4, n // 4, seed)
    to, tg, so, sr = inputs.uneven_tasks(n, tasks, seed + 1, (1, 100), s_range)
    return x, to, tg, so, sr


def submit(pool, to, tg, so, sr):
    return pool.submit_csr(np.zeros(len(to) - 1, np.uint32), to, tg, so, sr)


@pytest.mark.parametrize("budget", [0, 64 << 10])
def test_replay_matches_capture_and_oracle(gc, orc, budget):
    x, to, tg, so, sr = uneven()
    n = x.shape[0]
    pool = make_pool(gc, torch, n, n, staging_budget_bytes=budget)
    ids = np.arange(n, dtype=np.uint32)
    pool.upload(ids, x)
    submit(pool, to, tg, so, sr)
    g = gc.Graph(pool)
    if budget:
        assert pool.stats()["last_waves"] > 1
    first = g.results()
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    assert per_task_errors(gc.value(first), ref, to).max() <= TOL
    tot1 = pool.totals(ids)
    g.launch()
    g.wait()
    again = g.results()
    assert np.array_equal(again, first)
    g.launch()
    g.wait()
    np.testing.assert_allclose(pool.totals(ids), 3 * tot1, rtol=1e-12, atol=1e-300)
    # values re-uploaded in place are read by the next replay
    x2 = inputs.drift(x, seed=77, sigma=1e-2)
    pool.upload(ids, x2)
    g.launch()
    g.wait()
    ref2 = orc.gravity_batch(x2, to, tg, so, sr, EPS2)
    assert per_task_errors(gc.value(g.results()), ref2, to).max() <= TOL
    g.close()
    pool.close()


def test_replay_refused_after_table_change(gc):
    x, to, tg, so, sr = uneven(n=8000, tasks=40)
    n = x.shape[0]
    pool = make_pool(gc, torch, 2 * n, 2 * n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    # the graph's batch references only the first half of the ids
    half = n // 2
    keep = (tg < half)
    to_h = np.zeros(len(to), np.uint64)
    so_h = np.zeros(len(so), np.uint64)
    tg_l, sr_l = [], []
    for t in range(len(to) - 1):
        a = tg[to[t]:to[t + 1]] % half
        b = sr[so[t]:so[t + 1]] % half
        tg_l.append(a)
        sr_l.append(b)
        to_h[t + 1] = to_h[t] + len(a)
        so_h[t + 1] = so_h[t] + len(b)
    submit(pool, to_h, np.concatenate(tg_l), so_h, np.concatenate(sr_l))
    g = gc.Graph(pool)
    g.launch()
    g.wait()
    # a batch of other ids assigns new slots: the graph is stale
    other = np.arange(half, n, dtype=np.uint32)
    pool.submit_csr(np.zeros(1, np.uint32), np.array([0, 8], np.uint64), other[:8],
                    np.array([0, 16], np.uint64), other[8:24])
    pool.flush()
    with pytest.raises(gc.GcError) as e:
        g.launch()
    assert e.value.code == gc.GC_ERR_STATE
    g.close()
    pool.close()
    assert keep.any()


def test_capture_needs_the_batch_to_fit(gc):
    x, to, tg, so, sr = uneven(n=6000, tasks=60, s_range=(1, 400))
    n = x.shape[0]
    # a pool for half the ids; waves of at most 1024 entries each fit it,
    # the whole batch does not
    pool = make_pool(gc, torch, n, n // 2, staging_budget_bytes=16 << 10)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    submit(pool, to, tg, so, sr)
    with pytest.raises(gc.GcError) as e:
        gc.Graph(pool)
    assert e.value.code in (gc.GC_ERR_POOL_FULL, gc.GC_ERR_BUDGET)
    with pytest.raises(gc.GcError) as e:
        gc.Graph(pool)                 # nothing pending
    assert e.value.code == gc.GC_ERR_STATE
    pool.close()


def test_lj_batch_replays(gc, orc):
    sysm = inputs.fcc_lj(8, inputs.SEED_BASE + 3, ncell=5)
    n = sysm.n
    pool = make_pool(gc, torch, n, n, lj_rc2=RC2, md_edge=sysm.edge)
    pool.upload(np.arange(n, dtype=np.uint32), sysm.u)
    pool.build_md(torch.from_numpy(sysm.cell.astype(np.int32)).cuda(), sysm.ncell)
    g = gc.Graph(pool)
    first = g.results()
    g.launch()
    g.wait()
    assert np.array_equal(g.results(), first)
    # sampled tasks against the oracle
    start, atoms = orc.md_cells(sysm.cell, sysm.ncell ** 3)
    ta, tb, td, ts = orc.md_tasks(sysm.ncell)
    cnt = (start[1:] - start[:-1]).astype(np.int64)
    roff = np.concatenate([[0], np.cumsum(cnt[ta] + np.where(ts != 0, 0, cnt[tb]))])
    vals = gc.value(first)
    for k in [0, 1, 13, len(ta) // 2, len(ta) - 1]:
        A = atoms[start[ta[k]]:start[ta[k] + 1]]
        B = atoms[start[tb[k]]:start[tb[k] + 1]]
        fa, fb = orc.lj(sysm.u, A, None if ts[k] else B, bool(ts[k]), td[k], sysm.E,
                        rc2_grid=RC2_GRID)
        ref = fa if ts[k] else np.concatenate([fa, fb])
        assert rel_l2(vals[roff[k]:roff[k + 1], :3], ref[:, :3]) <= TOL, k
    g.close()
    pool.close()
