"""Shared helpers of the GPU parity tests (imported by tests only)."""
import numpy as np

EPS2 = float(np.float32(1e-4))   # softening 0.01, as an exact float32 value
TOL = 1e-5                       # per-result relative L2 force error
S21 = float(1 << 21)
RC2 = 6.25                       # (2.5 sigma)^2, on the 2^-42 grid
RC2_GRID = int(RC2 * S21 * S21)


def rel_l2(got, ref):
    """Relative L2 error; exact zero required when the reference is zero."""
    nr = np.linalg.norm(ref)
    if nr < 1e-30:
        return 0.0 if np.linalg.norm(got) == 0 else np.inf
    return float(np.linalg.norm(got - ref) / nr)


def per_task_errors(got_rows, ref_rows, row_off):
    """e_r over the force components (first 3) of each task's rows."""
    errs = []
    for t in range(len(row_off) - 1):
        a, b = int(row_off[t]), int(row_off[t + 1])
        if b == a:
            continue
        errs.append(rel_l2(got_rows[a:b, :3], ref_rows[a:b, :3]))
    return np.array(errs)


def make_pool(gcharm, torch, id_cap, cap, **kw):
    stream = torch.cuda.current_stream().cuda_stream
    kw.setdefault("eps2", EPS2)
    return gcharm.Pool(id_capacity=id_cap, pool_capacity=cap, stream=stream, **kw)
