"""Pins for the oracle's planar MD case (the paper's MD runs in two
dimensions, Section 4.2): the task list covers every pair of neighbouring
cells once, and per-atom forces, energies and the count of pairs inside the
cutoff summed over the tasks equal a brute-force minimum-image pair sum."""
import numpy as np

from paper_2008_05712_gb300 import inputs

S = float(1 << 21)
RC = 2.5
RC2_GRID = int(RC * RC * S * S)


def test_task_coverage(orc):
    for m in (3, 4, 7):
        a, b, d, s = orc.md_tasks_2d(m)
        assert len(a) == 5 * m * m and int(s.sum()) == m * m
        assert np.all(d[:, 2] == 0)
        pairs = set()
        for k in range(len(a)):
            if s[k]:
                assert a[k] == b[k] and not d[k].any()
                continue
            x, y = a[k] % m, a[k] // m
            assert b[k] == (x + d[k, 0]) % m + m * ((y + d[k, 1]) % m)
            key = (min(a[k], b[k]), max(a[k], b[k]), )
            # an unordered pair of cells may be neighbours through two
            # images only when m < 3; here each appears once
            assert key not in pairs or m < 3
            pairs.add(key)
        # every cell has 8 distinct neighbours: 4 m^2 unordered pairs
        assert len(pairs) == 4 * m * m


def brute_force(sysm):
    m, E = sysm.ncell, sysm.E
    c = sysm.cell.astype(np.int64)
    X = np.stack([c % m, c // m], 1) * E + sysm.U[:, :2]
    L = m * E
    n = sysm.n
    F = np.zeros((n, 2))
    U = np.zeros(n)
    inside = 0
    for i in range(n):
        d = X - X[i]                                 # x_j - x_i, grid units
        d -= L * np.rint(d / L).astype(np.int64)
        r2g = (d * d).sum(1)
        sel = (r2g < RC2_GRID) & (np.arange(n) != i)
        inside += int(sel[i + 1:].sum())
        r = d[sel] / S
        r2 = (r * r).sum(1)
        s6 = (1.0 / r2) ** 3
        coef = 24.0 * (2.0 * s6 * s6 - s6) / r2
        F[i] = -(coef[:, None] * r).sum(0)
        U[i] = 0.5 * (4.0 * (s6 * s6 - s6)).sum()
    return F, U, inside


def test_tasks_equal_brute_force(orc):
    sysm = inputs.lj_2d(12, inputs.SEED_BASE + 5, ncell=5)      # edge 2.86 >= rc
    assert sysm.E / S >= RC
    start, atoms = orc.md_cells(sysm.cell, sysm.ncell ** 2)
    ta, tb, td, ts = orc.md_tasks_2d(sysm.ncell)
    F = np.zeros((sysm.n, 4))
    for k in range(len(ta)):
        A = atoms[start[ta[k]]:start[ta[k] + 1]]
        B = atoms[start[tb[k]]:start[tb[k] + 1]]
        fa, fb = orc.lj(sysm.u, A, None if ts[k] else B, bool(ts[k]), td[k], sysm.E,
                        rc2_grid=RC2_GRID)
        F[A] += fa
        if not ts[k]:
            F[B] += fb
    Fb, Ub, _ = brute_force(sysm)
    assert np.all(F[:, 2] == 0)
    np.testing.assert_allclose(F[:, :2], Fb, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(F[:, 3], Ub, rtol=1e-12, atol=1e-12)
    # momentum: the forces sum to zero
    assert np.abs(F[:, :2].sum(0)).max() < 1e-9
