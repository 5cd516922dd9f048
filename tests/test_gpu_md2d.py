"""GPU parity of the planar MD case (the paper's MD is two-dimensional,
Section 4.2) against the FP64 oracle: cells and task list bit-exact, cutoff
decisions exact, forces within the per-result tolerance, Newton III per
task, per-atom totals."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import RC2, RC2_GRID, TOL, make_pool, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    return gcharm


@pytest.mark.parametrize("side,ncell", [(40, 13), (128, 42)])
def test_planar_md_vs_oracle(gc, orc, side, ncell):
    sysm = inputs.lj_2d(side, inputs.SEED_BASE + 6, ncell=ncell)
    assert sysm.E / float(1 << 21) >= 2.5
    n, m = sysm.n, sysm.ncell
    pool = make_pool(gc, torch, n, n, lj_rc2=RC2, md_edge=sysm.edge)
    pool.upload(np.arange(n, dtype=np.uint32), sysm.u)
    info = pool.build_md(torch.from_numpy(sysm.cell.astype(np.int32)).cuda(), m, dim=2)
    pool.flush()
    start, atoms = pool.md_cells(n, m, dim=2)
    s0, a0 = orc.md_cells(sysm.cell, m * m)
    assert np.array_equal(start, s0) and np.array_equal(atoms, a0)
    ta, tb, td, ts = orc.md_tasks_2d(m)
    assert info["tasks"] == len(ta) == 5 * m * m
    got = pool.values()
    row, errs, inside = 0, [], 0
    tot_ref = np.zeros((n, 4))
    for k in range(len(ta)):
        A = a0[s0[ta[k]]:s0[ta[k] + 1]]
        B = a0[s0[tb[k]]:s0[tb[k] + 1]]
        fa, fb = orc.lj(sysm.u, A, None if ts[k] else B, bool(ts[k]), td[k], sysm.E,
                        rc2_grid=RC2_GRID)
        ref = fa if ts[k] else np.concatenate([fa, fb])
        g = got[row:row + len(ref)]
        row += len(ref)
        errs.append(rel_l2(g[:, :3], ref[:, :3]))
        assert np.all(g[:, 2] == 0)
        assert np.max(np.abs(g[:, :2].sum(axis=0))) <= 1e-5 * max(np.abs(g[:, :2]).sum(), 1e-30)
        tot_ref[A] += fa
        if not ts[k]:
            tot_ref[B] += fb
    assert row == got.shape[0]
    assert max(errs) <= TOL, max(errs)
    tot = pool.totals(np.arange(n, dtype=np.uint32))
    assert rel_l2(tot[:, :2], tot_ref[:, :2]) <= TOL
    # pairs inside the cutoff: brute force on the integer grid
    c = sysm.cell.astype(np.int64)
    X = np.stack([c % m, c // m], 1) * sysm.E + sysm.U[:, :2]
    L = m * sysm.E
    cnt = 0
    for i in range(n):
        d = X[i + 1:] - X[i]
        d -= L * np.rint(d / L).astype(np.int64)
        cnt += int(((d * d).sum(1) < RC2_GRID).sum())
    assert pool.stats()["lj_pairs_in_cutoff"] == cnt
    pool.close()
