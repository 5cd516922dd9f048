"""The no-allocation gravity entry point, checked against the FP64 oracle.

Some callers cannot allocate device memory at the moment they need a
result: code inside a framework whose caching allocator already holds the
device memory budget, and latency-critical serving threads that cannot take
the device-wide synchronisation of cudaMalloc/cudaFree.  gc_gravity_noalloc
serves them from one fixed scratch array.  Its results must match the
oracle's softened gravity within the force tolerance on two calls in a row
(the scratch keeps the previous call's contents) and agree with the regular
pool path; a call with inconsistent offsets must say so in its output (NaN
rows) rather than leave stale rows behind.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import EPS2, TOL, make_pool, per_task_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def _values(rows):
    """FP64 value s - c of compensated rows (n, 8) -> (n, 4)."""
    return rows[:, :4].astype(np.float64) - rows[:, 4:].astype(np.float64)


def _case(seed, n_tasks, n_ids=12000):
    x = inputs.merger(9000, 3000, seed)
    to, tg, so, sr = inputs.uneven_tasks(n_ids, n_tasks, seed + 1, (1, 70), (1, 5000))
    return x, to, tg, so, sr


def test_noalloc_matches_oracle_on_two_calls():
    from oracle import oracle as O
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    for call, (seed, n_tasks) in enumerate([(41, 150), (42, 90)]):
        x, to, tg, so, sr = _case(seed, n_tasks)
        ref = O.gravity_batch(x, to, tg, so, sr, np.float32(EPS2))
        out = torch.full((len(tg), 8), float("nan"), dtype=torch.float32, device="cuda")
        gcharm.gravity_noalloc(_dev(to), _dev(x[tg]), _dev(so), _dev(x[sr]), len(tg), EPS2,
                               out)
        torch.cuda.synchronize()
        got = _values(out.cpu().numpy())
        assert np.all(np.isfinite(got)), call
        errs = per_task_errors(got, ref, to)
        assert errs.max() <= TOL, (call, errs.max())


def test_noalloc_agrees_with_regular_path():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    n_ids = 12000
    x, to, tg, so, sr = _case(43, 120, n_ids)
    pool = make_pool(gcharm, torch, n_ids, n_ids)
    pool.upload(np.arange(n_ids, dtype=np.uint32), x)
    pool.submit_csr(np.zeros(len(to) - 1, np.uint32), to, tg, so, sr)
    pool.flush()
    ref = _values(pool.results())
    pool.close()
    out = torch.empty((len(tg), 8), dtype=torch.float32, device="cuda")
    gcharm.gravity_noalloc(_dev(to), _dev(x[tg]), _dev(so), _dev(x[sr]), len(tg), EPS2, out)
    torch.cuda.synchronize()
    assert per_task_errors(_values(out.cpu().numpy()), ref, to).max() <= TOL


def test_noalloc_bad_offsets_give_nan_rows_then_recovers():
    from oracle import oracle as O
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    x, to, tg, so, sr = _case(44, 40)
    tgt, src = _dev(x[tg]), _dev(x[sr])
    n = len(tg)
    # the offsets end one short of the target total the caller states
    bad = to.copy()
    bad[-1] -= 1
    out = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    gcharm.gravity_noalloc(_dev(bad), tgt, _dev(so), src, n, EPS2, out)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    # decreasing offsets
    dec = to.copy()
    dec[5], dec[6] = dec[6], dec[5]
    out.zero_()
    if dec[5] != dec[6]:
        gcharm.gravity_noalloc(_dev(dec), tgt, _dev(so), src, n, EPS2, out)
        torch.cuda.synchronize()
        assert torch.isnan(out).all()
    # the next consistent call is unaffected
    gcharm.gravity_noalloc(_dev(to), tgt, _dev(so), src, n, EPS2, out)
    torch.cuda.synchronize()
    ref = O.gravity_batch(x, to, tg, so, sr, np.float32(EPS2))
    assert per_task_errors(_values(out.cpu().numpy()), ref, to).max() <= TOL


def test_noalloc_allocates_nothing_after_set_up():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    x, to, tg, so, sr = _case(45, 60)
    args = (_dev(to), _dev(x[tg]), _dev(so), _dev(x[sr]), len(tg), EPS2)
    out = torch.empty((len(tg), 8), dtype=torch.float32, device="cuda")
    gcharm.gravity_noalloc(*args, out)          # first call: set-up, kernels loaded
    torch.cuda.synchronize()
    first = out.clone()
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        gcharm.gravity_noalloc(*args, out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, first)              # the same rows, call after call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    n = gcharm.NOALLOC_MAX_TARGETS + 1
    off = _dev(np.array([0, n], np.uint64))
    x = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(gcharm.GcError) as e:
        gcharm.gravity_noalloc(off, x, off, x, n, EPS2, out)
    assert e.value.code == gcharm.GC_ERR_TOO_LARGE


def test_noalloc_binding_rejects_mismatched_tensors():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    off = _dev(np.array([0, 4], np.uint64))
    x = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):          # 32-bit offsets
        gcharm.gravity_noalloc(off.to(torch.int32), x, off, x, 4, EPS2, out)
    with pytest.raises(ValueError):          # too few target rows
        gcharm.gravity_noalloc(off, x[:3], off, x, 4, EPS2, out)
    with pytest.raises(ValueError):          # output of the wrong shape
        gcharm.gravity_noalloc(off, x, off, x, 4, EPS2, out[:3])
    with pytest.raises(ValueError):          # host tensor
        gcharm.gravity_noalloc(off, x.cpu(), off, x, 4, EPS2, out)
