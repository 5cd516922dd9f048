"""GPU tests of the serving loop (Section 3.1: work requests combined as
they arrive, while earlier batches run on the device): every task's
result is the same in the mix as alone, both within the per-result
tolerance of the FP64 oracle; policies, admission by the staging budget and
the latency report."""
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


def workload(n_ids=32768, n_tasks=600, seed=41, t_range=(8, 256), s_range=(16, 4096)):
    x = inputs.merger(3 * n_ids // 4, n_ids // 4, seed)
    to, tg, so, sr = inputs.uneven_tasks(n_ids, n_tasks, seed + 1, t_range, s_range)
    return x, to, tg, so, sr


def serve(gc, pool, to, tg, so, sr, arrivals, **kw):
    kinds = np.zeros(len(to) - 1, np.uint32)
    return pool.serve(arrivals, kinds, to, tg, so, sr, want_results=True, **kw)


def check_report(rep, lat, to, so):
    n = len(to) - 1
    nt = (to[1:] - to[:-1]).astype(np.int64)
    ns = (so[1:] - so[:-1]).astype(np.int64)
    assert rep["tasks"] == n
    assert rep["interactions"] == int((nt * ns).sum())
    assert lat.shape[0] == n and (lat > 0).all()
    assert rep["lat_p50_us"] <= rep["lat_p99_us"] <= rep["lat_max_us"] + 1e-9
    assert rep["lat_max_us"] == pytest.approx(lat.max() * 1e-3)
    assert rep["batches"] >= 1 and rep["mean_batch"] == pytest.approx(n / rep["batches"])


def test_serve_mix_equals_alone_and_oracle(gc, orc):
    x, to, tg, so, sr = workload()
    n = x.shape[0]
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    arr = inputs.poisson_arrivals(len(to) - 1, 2e4, 7)
    rep, lat, rows = serve(gc, pool, to, tg, so, sr, arr,
                           policy=gc.GC_COMBINE_GREEDY, max_in_flight=2)
    check_report(rep, lat, to, so)
    assert rep["batches"] >= 2
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    mix = gc.value(rows)
    errs = per_task_errors(mix, ref, to)
    assert errs.max() <= TOL, errs.max()
    # per-id FP64 totals accumulated over every served batch
    tot_ref = orc.reduce(tg, ref, n)
    u = np.unique(tg)
    assert rel_l2(pool.totals(u)[:, :3], tot_ref[u, :3]) <= TOL
    # each sampled task alone: its own batch of one
    g = np.random.default_rng(5)
    for t in sorted(g.choice(len(to) - 1, 40, replace=False)):
        a, b = int(to[t]), int(to[t + 1])
        c, d = int(so[t]), int(so[t + 1])
        one_to = np.array([0, b - a], np.uint64)
        one_so = np.array([0, d - c], np.uint64)
        bi = pool.submit_csr(np.zeros(1, np.uint32), one_to, tg[a:b], one_so, sr[c:d])
        pool.flush()
        pool.wait(bi)
        alone = pool.values()
        assert rel_l2(mix[a:b, :3], alone[:, :3]) <= TOL
        assert rel_l2(alone[:, :3], ref[a:b, :3]) <= TOL
    pool.close()


def test_serve_policies(gc, orc):
    x, to, tg, so, sr = workload(n_ids=8192, n_tasks=95, seed=43, s_range=(16, 1024))
    n = x.shape[0]
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    arr = inputs.poisson_arrivals(len(to) - 1, 5e3, 9)
    for policy, extra in [(gc.GC_COMBINE_PER_TASK, {}),
                          (gc.GC_COMBINE_STATIC, {"static_n": 10}),
                          (gc.GC_COMBINE_ADAPTIVE, {}),
                          (gc.GC_COMBINE_ADAPTIVE, {"max_size": 7}),
                          (gc.GC_COMBINE_ADAPTIVE_WINDOW, {"max_size": 16, "window": 32}),
                          (gc.GC_COMBINE_GREEDY, {"max_size": 5})]:
        for inflight in (1, 2):
            pool = make_pool(gc, torch, n, n)
            pool.upload(np.arange(n, dtype=np.uint32), x)
            rep, lat, rows = serve(gc, pool, to, tg, so, sr, arr, policy=policy,
                                   max_in_flight=inflight, **extra)
            check_report(rep, lat, to, so)
            if policy == gc.GC_COMBINE_PER_TASK:
                assert rep["batches"] == len(to) - 1
            if extra.get("max_size"):
                m = extra["max_size"]
                assert rep["batches"] >= (len(to) - 1 + m - 1) // m
            errs = per_task_errors(gc.value(rows), ref, to)
            assert errs.max() <= TOL, (policy, inflight, errs.max())
            pool.close()


def test_serve_admission_by_budget(gc, orc):
    x, to, tg, so, sr = workload(n_ids=8192, n_tasks=120, seed=45, s_range=(16, 2048))
    n = x.shape[0]
    nt = (to[1:] - to[:-1]).astype(np.int64)
    ns = (so[1:] - so[:-1]).astype(np.int64)
    budget = int(((nt + ns) * 16).max() * 2)
    pool = make_pool(gc, torch, n, n, staging_budget_bytes=budget)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    # all requests at once: the combiner would take them all; the budget
    # splits them into batches of the oldest requests that fit
    arr = np.zeros(len(to) - 1, np.uint64)
    rep, lat, rows = serve(gc, pool, to, tg, so, sr, arr, policy=gc.GC_COMBINE_ADAPTIVE,
                           max_size=1 << 20)
    check_report(rep, lat, to, so)
    min_batches = int(np.ceil((nt + ns).sum() * 16 / budget))
    assert rep["batches"] >= min_batches
    assert pool.stats()["last_waves"] == 1     # admission kept each batch in budget
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    errs = per_task_errors(gc.value(rows), ref, to)
    assert errs.max() <= TOL, errs.max()
    pool.close()


def test_serve_rejects(gc):
    x, to, tg, so, sr = workload(n_ids=4096, n_tasks=4, seed=47, s_range=(16, 64))
    n = x.shape[0]
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    kinds = np.zeros(4, np.uint32)
    with pytest.raises(gc.GcError) as e:
        pool.serve(np.array([5, 4, 6, 7], np.uint64), kinds, to, tg, so, sr)
    assert e.value.code == gc.GC_ERR_ARG
    with pytest.raises(gc.GcError) as e:
        pool.serve(np.zeros(4, np.uint64), kinds, to, tg, so, sr, max_in_flight=3)
    assert e.value.code == gc.GC_ERR_ARG
    pool.submit_csr(kinds[:1], to[:2], tg, so[:2], sr)
    with pytest.raises(gc.GcError) as e:
        pool.serve(np.zeros(4, np.uint64), kinds, to, tg, so, sr)
    assert e.value.code == gc.GC_ERR_STATE
    pool.flush()
    rep, lat, _ = pool.serve(np.zeros(0, np.uint64), kinds[:0], to[:1], tg[:0], so[:1], sr[:0])
    assert rep["tasks"] == 0 and lat.shape[0] == 0
    pool.close()


def test_serve_cycled_task_set_warmup_and_drain(gc):
    """A task set replayed cyclically (arrival k runs task k mod m), the
    warm-up arrivals left out of the latency statistics, and an overloaded
    run (one task per batch at 1e6 tasks/s) cut off by the drain limit with
    the rest reported unserved."""
    x, to, tg, so, sr = workload(n_tasks=200)
    n_ids = x.shape[0]
    pool = make_pool(gc, torch, n_ids, n_ids)
    pool.upload(np.arange(n_ids, dtype=np.uint32), x)
    m, n = 200, 1000
    kinds = np.zeros(m, np.uint32)
    nt = (to[1:] - to[:-1]).astype(np.int64)
    ns = (so[1:] - so[:-1]).astype(np.int64)
    arr = inputs.poisson_arrivals(n, 5e4, 9)
    warm = int(arr[199])
    rep, lat, _ = pool.serve(arr, kinds, to, tg, so, sr, policy=gc.GC_COMBINE_GREEDY,
                             task_set=m, warmup_ns=warm)
    k = np.arange(n) % m
    assert rep["interactions"] == int((nt[k] * ns[k]).sum())
    assert rep["unserved"] == 0
    assert rep["measured"] == int((arr >= warm).sum())
    assert (lat != np.iinfo(np.uint64).max).all()
    # results of a cycled set are refused (rows would repeat)
    with pytest.raises(gc.GcError):
        pool.serve(arr, kinds, to, tg, so, sr, task_set=m, want_results=True)
    # overload: the queue left after the schedule is not drained past the limit
    arr2 = inputs.poisson_arrivals(20000, 1e6, 10)          # about 20 ms of arrivals
    rep2, lat2, _ = pool.serve(arr2, kinds, to, tg, so, sr, policy=gc.GC_COMBINE_PER_TASK,
                               task_set=m, drain_ns=50_000_000)
    served = lat2 != np.iinfo(np.uint64).max
    assert rep2["unserved"] > 0 and int((~served).sum()) == rep2["unserved"]
    assert rep2["wall_s"] < 2.0
    assert rep2["measured"] == int(served.sum()) and rep2["batches"] == int(served.sum())
    pool.close()
