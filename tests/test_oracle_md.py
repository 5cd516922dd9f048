"""Pins for the oracle's MD cells, cell-pair tasks and Lennard-Jones pair
interaction (Section 4.2: patches own particles; a compute object's
interact() updates the forces of the particles of both patches)."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs

S = float(1 << 21)
RC2_GRID = int(2.5 * 2.5 * S * S)   # rc = 2.5 sigma, on the 2^-21 grid


def two_atoms(dx, dy=0.0, dz=0.0, d3=(0, 0, 0), E=None):
    """Atom 0 at local (0.5, 0.5, 0.5) of cell A, atom 1 at offset (dx,dy,dz)
    from it, expressed in cell B = A + d3 of edge E."""
    E = E if E is not None else int(3 * S)
    edge = E / S
    u0 = np.array([0.5, 0.5, 0.5])
    u1 = u0 + np.array([dx, dy, dz]) - np.array(d3) * edge
    t = np.array([[*u0, 1.0], [*u1, 1.0]], np.float32)
    assert np.all(t[1, :3].astype(np.float64) == u1)   # exact on the grid
    return t, E


def test_force_at_sigma(orc):
    # r = sigma: |F| = 24 eps / sigma; repulsive (atom 0 pushed to -x); U = 0
    t, E = two_atoms(1.0)
    a, b = orc.lj(t, [0], [1], False, (0, 0, 0), E, rc2_grid=RC2_GRID)
    assert a[0, 0] == pytest.approx(-24.0, rel=1e-15)
    assert a[0, 1] == 0 and a[0, 2] == 0 and a[0, 3] == 0
    np.testing.assert_array_equal(b[0, :3], -a[0, :3])


def test_energy_minimum(orc):
    # r = 2^(1/6) sigma (nearest grid point): U = -eps, F ~ 0
    r = round(2 ** (1 / 6) * S) / S
    t, E = two_atoms(r)
    a, b = orc.lj(t, [0], [1], False, (0, 0, 0), E, rc2_grid=RC2_GRID)
    assert a[0, 3] + b[0, 3] == pytest.approx(-1.0, abs=1e-9)
    # |dF/dr| at the minimum is 57.1 eps/sigma^2; grid error <= 2^-22
    assert abs(a[0, 0]) < 57.2 * 2 ** -22


def test_attractive_tail_and_cutoff(orc):
    # r = 2: U = 4 (2^-12 - 2^-6), F = 24 (2 2^-12 - 2^-6)/2 (attractive)
    t, E = two_atoms(2.0)
    a, _ = orc.lj(t, [0], [1], False, (0, 0, 0), E, rc2_grid=RC2_GRID)
    assert a[0, 0] == pytest.approx(-24 * (2 * 2 ** -12 - 2 ** -6) / 2, rel=1e-15)
    assert a[0, 3] == pytest.approx(0.5 * 4 * (2 ** -12 - 2 ** -6), rel=1e-15)
    # exactly at the cutoff: excluded; one grid step inside: included
    t, E = two_atoms(2.5)
    a, b = orc.lj(t, [0], [1], False, (0, 0, 0), E, rc2_grid=RC2_GRID)
    assert np.all(a == 0) and np.all(b == 0)
    t, E = two_atoms(2.5 - 1 / S)
    a, _ = orc.lj(t, [0], [1], False, (0, 0, 0), E, rc2_grid=RC2_GRID)
    # attractive: atom 0 pulled towards +x; |F(rc)| = 24 (2 s^12 - s^6)/rc ~ 0.039
    assert a[0, 0] == pytest.approx(-24 * (2 * 0.4 ** 12 - 0.4 ** 6) / 2.5, rel=1e-5)


def test_image_offset(orc):
    # the same physical pair written through a neighbour cell offset gives the
    # same force: B = A + (1, 0, -1)
    t0, E = two_atoms(1.25, 0.5, -0.75)
    t1, _ = two_atoms(1.25, 0.5, -0.75, d3=(1, 0, -1), E=E)
    a0, b0 = orc.lj(t0, [0], [1], False, (0, 0, 0), E, rc2_grid=RC2_GRID)
    a1, b1 = orc.lj(t1, [0], [1], False, (1, 0, -1), E, rc2_grid=RC2_GRID)
    np.testing.assert_array_equal(a0, a1)
    np.testing.assert_array_equal(b0, b1)


def test_self_task_pairs_once(orc):
    # self task over 3 atoms == the three pair tasks summed
    rows = np.array([[0.5, 0.5, 0.5, 1], [1.5, 0.5, 0.5, 1], [0.5, 1.75, 0.5, 1]],
                    np.float32)
    E = int(3 * S)
    a, _ = orc.lj(rows, [0, 1, 2], None, True, (0, 0, 0), E, rc2_grid=RC2_GRID)
    tot = np.zeros((3, 4))
    for i, j in [(0, 1), (0, 2), (1, 2)]:
        x, y = orc.lj(rows, [i], [j], False, (0, 0, 0), E, rc2_grid=RC2_GRID)
        tot[i] += x[0]
        tot[j] += y[0]
    np.testing.assert_allclose(a, tot, rtol=1e-15, atol=1e-15)
    assert np.max(np.abs(a[:, :3].sum(axis=0))) < 1e-13


def test_cells_and_tasks(orc):
    m = 4
    a, b, d, s = orc.md_tasks(m)
    assert len(a) == 14 * m ** 3
    # every unordered pair of neighbouring cells (and every cell with itself)
    # appears exactly once
    seen = {}
    for k in range(len(a)):
        key = (min(a[k], b[k]), max(a[k], b[k]), s[k])
        if s[k]:
            assert a[k] == b[k] and tuple(d[k]) == (0, 0, 0)
        seen[key] = seen.get(key, 0) + 1
    assert all(v == 1 for v in seen.values())
    def xyz(c):
        return np.array([c % m, (c // m) % m, c // (m * m)])
    for k in range(len(a)):
        if not s[k]:
            assert np.all((xyz(a[k]) + d[k]) % m == xyz(b[k]))
    # cell grouping = stable argsort of the cell index
    cell = inputs.rng(5).integers(0, m ** 3, 500).astype(np.uint32)
    start, atoms = orc.md_cells(cell, m ** 3)
    assert np.array_equal(atoms, np.argsort(cell, kind="stable"))
    assert np.array_equal(np.diff(start.astype(np.int64)), np.bincount(cell, minlength=m ** 3))


def run_all_tasks(orc, sysm):
    m = sysm.ncell
    start, atoms = orc.md_cells(sysm.cell, m ** 3)
    ta, tb, td, ts = orc.md_tasks(m)
    tot = np.zeros((sysm.n, 4))
    for k in range(len(ta)):
        A = atoms[start[ta[k]]:start[ta[k] + 1]]
        B = atoms[start[tb[k]]:start[tb[k] + 1]]
        fa, fb = orc.lj(sysm.u, A, None if ts[k] else B, bool(ts[k]), td[k], sysm.E,
                        rc2_grid=RC2_GRID)
        tot[A] += fa
        if not ts[k]:
            tot[B] += fb
    return tot


def test_perfect_fcc_lattice(orc):
    # FCC lattice with constant 1.75 (all sites on the 2^-21 grid), 12^3
    # unit cells in an 8^3 grid of MD cells of edge 2.625 >= rc.  By symmetry
    # every atom feels zero force, and every atom's energy is the lattice sum
    # over the neighbour shells inside rc: 12 at a/sqrt2, 6 at a,
    # 24 at a sqrt(3/2), 12 at a sqrt2.
    a_lat, nl, m = 1.75, 12, 8
    E = int(21.0 / m * S)
    base = np.array([[0, 0, 0], [.5, .5, 0], [.5, 0, .5], [0, .5, .5]])
    g = np.stack(np.meshgrid(*[np.arange(nl)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = ((g[:, None, :] + base[None]) * a_lat).reshape(-1, 3)
    X = np.rint(pos * S).astype(np.int64)
    C = X // E
    U = X - C * E
    cell = (C[:, 0] + m * (C[:, 1] + m * C[:, 2])).astype(np.uint32)
    sysm = inputs.MDSystem(cell, U, E, m)
    tot = run_all_tasks(orc, sysm)
    assert np.max(np.abs(tot[:, :3])) < 1e-12

    def u(r):
        return 4 * (r ** -12 - r ** -6)
    shells = [(12, a_lat / np.sqrt(2)), (6, a_lat), (24, a_lat * np.sqrt(1.5)),
              (12, a_lat * np.sqrt(2))]
    expect = 0.5 * sum(n * u(r) for n, r in shells)
    np.testing.assert_allclose(tot[:, 3], expect, rtol=1e-12)


def test_newton_per_task_jittered(orc):
    sysm = inputs.fcc_lj(6, 3, ncell=4)   # edge 2.52 >= rc
    m = sysm.ncell
    start, atoms = orc.md_cells(sysm.cell, m ** 3)
    ta, tb, td, ts = orc.md_tasks(m)
    for k in range(0, len(ta), 7):
        A = atoms[start[ta[k]]:start[ta[k] + 1]]
        B = atoms[start[tb[k]]:start[tb[k] + 1]]
        fa, fb = orc.lj(sysm.u, A, None if ts[k] else B, bool(ts[k]), td[k], sysm.E,
                        rc2_grid=RC2_GRID)
        net = fa[:, :3].sum(axis=0) + (0 if ts[k] else fb[:, :3].sum(axis=0))
        scale = np.abs(fa[:, :3]).sum() + (0 if ts[k] else np.abs(fb[:, :3]).sum())
        assert np.max(np.abs(net)) <= 1e-13 * max(scale, 1e-300)
