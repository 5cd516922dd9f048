"""The no-allocation gravity entry point against the regular entry point.

Some callers cannot allocate device memory at the moment they need a
result: code that runs while a stream is being captured into a CUDA graph,
code inside a framework whose allocator owns the device memory, and
latency-critical serving threads that cannot take the device-wide
synchronisation of cudaMalloc/cudaFree.  gc_gravity_noalloc serves them
from one fixed scratch array.  Its results must match the regular pool path
(upload, submit, flush) within the force tolerance, on two calls in a row,
since the scratch keeps the previous call's contents.

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


def test_noalloc_matches_regular_path_on_two_calls():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    for call, (seed, n_tasks) in enumerate([(41, 150), (42, 90)]):
        n_ids = 12000
        x = inputs.merger(9000, 3000, seed)
        to, tg, so, sr = inputs.uneven_tasks(n_ids, n_tasks, seed + 1, (1, 70), (1, 5000))
        # regular entry point
        pool = make_pool(gcharm, torch, n_ids, n_ids)
        pool.upload(np.arange(n_ids, dtype=np.uint32), x)
        pool.submit_csr(np.zeros(len(to) - 1, np.uint32), to, tg, so, sr)
        pool.flush()
        ref = gcharm.value(pool.results())
        pool.close()
        # no-allocation entry point on the same values, gathered in CSR order
        out = torch.full((len(tg), 8), float("nan"), dtype=torch.float32, device="cuda")
        gcharm.gravity_noalloc(_dev(to), _dev(x[tg]), _dev(so), _dev(x[sr]), len(tg), EPS2,
                               out)
        torch.cuda.synchronize()
        got = gcharm.value(out.cpu().numpy())
        assert np.all(np.isfinite(got)), call
        errs = per_task_errors(got, ref, to)
        assert errs.max() <= TOL, (call, errs.max())


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
