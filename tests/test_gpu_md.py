"""GPU parity of the MD path (Section 4.2: cell-pair compute objects update
both cells) against the FP64 oracle: cells bit-exact, cutoff decisions
exact, forces within 1e-5 relative L2 per task, Newton III per task."""
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


def run_md(gc, sysm, per_task=False):
    n = sysm.n
    pool = make_pool(gc, torch, n, n, lj_rc2=RC2, md_edge=sysm.edge)
    pool.upload(np.arange(n, dtype=np.uint32), sysm.u)
    info = pool.build_md(torch.from_numpy(sysm.cell.astype(np.int32)).cuda(), sysm.ncell)
    if per_task:
        pool.flush_per_task()
    else:
        pool.flush()
    return pool, info


@pytest.fixture(scope="module")
def small_md():
    # 8^3 FCC unit cells (2048 atoms), 5^3 MD cells of edge 2.687 >= 2.5
    return inputs.fcc_lj(8, inputs.SEED_BASE + 3, ncell=5)


def oracle_tasks(orc, sysm):
    m = sysm.ncell
    start, atoms = orc.md_cells(sysm.cell, m ** 3)
    ta, tb, td, ts = orc.md_tasks(m)
    return start, atoms, ta, tb, td, ts


def test_cells_bit_exact(gc, orc, small_md):
    pool, info = run_md(gc, small_md)
    start, atoms = pool.md_cells(small_md.n, small_md.ncell)
    s0, a0, ta, tb, td, ts = oracle_tasks(orc, small_md)
    assert np.array_equal(start, s0) and np.array_equal(atoms, a0)
    assert info["tasks"] == len(ta)
    pool.close()


def test_forces_vs_oracle(gc, orc, small_md):
    sysm = small_md
    pool, info = run_md(gc, sysm)
    got = pool.values()
    start, atoms, ta, tb, td, ts = oracle_tasks(orc, sysm)
    row = 0
    errs = []
    tot_ref = np.zeros((sysm.n, 4))
    in_cut = 0
    for k in range(len(ta)):
        A = atoms[start[ta[k]]:start[ta[k] + 1]]
        B = atoms[start[tb[k]]:start[tb[k] + 1]]
        fa, fb = orc.lj(sysm.u, A, None if ts[k] else B, bool(ts[k]), td[k], sysm.E,
                        rc2_grid=RC2_GRID)
        ref = fa if ts[k] else np.concatenate([fa, fb])
        g = got[row:row + len(ref)]
        row += len(ref)
        errs.append(rel_l2(g[:, :3], ref[:, :3]))
        tot_ref[A] += fa
        if not ts[k]:
            tot_ref[B] += fb
        # Newton III inside the task (both sides computed with the same ops)
        assert np.max(np.abs(g[:, :3].sum(axis=0))) <= 1e-5 * max(np.abs(g[:, :3]).sum(), 1e-30)
    assert row == got.shape[0]
    errs = np.array(errs)
    assert errs.max() <= TOL, errs.max()
    tot = pool.totals(np.arange(sysm.n, dtype=np.uint32))
    assert rel_l2(tot[:, :3], tot_ref[:, :3]) <= TOL
    np.testing.assert_allclose(tot[:, 3], tot_ref[:, 3], rtol=1e-5, atol=1e-6)
    pool.close()


def test_pairs_in_cutoff_exact(gc, orc, small_md):
    # count pairs within rc by brute force on the integer grid (minimum image)
    sysm = small_md
    pool, _ = run_md(gc, sysm)
    m, E = sysm.ncell, sysm.E
    c = sysm.cell.astype(np.int64)
    C3 = np.stack([c % m, (c // m) % m, c // (m * m)], 1)
    X = C3 * E + sysm.U
    L = m * E
    cnt = 0
    for i in range(sysm.n):
        d = X[i + 1:] - X[i]
        d -= L * np.rint(d / L).astype(np.int64)
        cnt += int(((d * d).sum(1) < RC2_GRID).sum())
    assert pool.stats()["lj_pairs_in_cutoff"] == cnt
    pool.close()


def test_perfect_lattice_zero_force(gc):
    # lattice constant 1.75 on the grid, 12^3 unit cells, 8^3 MD cells
    S = float(1 << 21)
    a_lat, nl, m = 1.75, 12, 8
    E = int(21.0 / m * S)
    base = np.array([[0, 0, 0], [.5, .5, 0], [.5, 0, .5], [0, .5, .5]])
    g = np.stack(np.meshgrid(*[np.arange(nl)] * 3, indexing="ij"), -1).reshape(-1, 3)
    X = np.rint(((g[:, None, :] + base[None]) * a_lat).reshape(-1, 3) * S).astype(np.int64)
    C = X // E
    sysm = inputs.MDSystem((C[:, 0] + m * (C[:, 1] + m * C[:, 2])).astype(np.uint32),
                           X - C * E, E, m)
    pool, _ = run_md(gc, sysm)
    tot = pool.totals(np.arange(sysm.n, dtype=np.uint32))
    # per-atom force ~0 against the scale of one nearest-neighbour force
    assert np.max(np.abs(tot[:, :3])) < 1e-4
    u = tot[:, 3]
    assert np.ptp(u) < 1e-5 * abs(u.mean())
    pool.close()


def test_per_task_launches_match(gc, small_md):
    p1, _ = run_md(gc, small_md)
    a = p1.results()
    p1.close()
    p2, _ = run_md(gc, small_md, per_task=True)
    b = p2.results()
    p2.close()
    assert np.array_equal(a, b)


def host_md_batch(gc, orc, sysm, dim=3):
    """The build's tasks as host CSR arrays (oracle cells and task list)."""
    m = sysm.ncell
    start, atoms = orc.md_cells(sysm.cell, m ** dim)
    ta, tb, td, ts = orc.md_tasks(m) if dim == 3 else orc.md_tasks_2d(m)
    tg = [atoms[start[a]:start[a + 1]] for a in ta]
    sr = [atoms[start[b]:start[b + 1]] if not s else atoms[:0] for b, s in zip(tb, ts)]
    to = np.zeros(len(ta) + 1, np.uint64)
    so = np.zeros(len(ta) + 1, np.uint64)
    to[1:] = np.cumsum([len(a) for a in tg])
    so[1:] = np.cumsum([len(a) for a in sr])
    kinds = np.where(ts != 0, gc.GC_LJ_SELF, gc.GC_LJ_PAIR).astype(np.uint32)
    return (kinds, to, np.concatenate(tg).astype(np.uint32), so,
            np.concatenate(sr).astype(np.uint32), td.astype(np.int8).reshape(-1))


@pytest.mark.parametrize("dim", [3, 2])
def test_cell_reduction_matches_sorted_path(gc, orc, small_md, dim):
    """A batch holding exactly one MD build sums each atom's rows per cell;
    the same tasks submitted from the host go through the general path (rows
    sorted by id).  Rows and per-atom totals agree bit for bit, over two
    consecutive batches (totals accumulate), and a build followed by another
    task in the same batch takes the general path."""
    sysm = small_md if dim == 3 else inputs.lj_2d(40, inputs.SEED_BASE + 6, ncell=13)
    n, m = sysm.n, sysm.ncell
    ids = np.arange(n, dtype=np.uint32)
    cell = torch.from_numpy(sysm.cell.astype(np.int32)).cuda()
    a = make_pool(gc, torch, n, n, lj_rc2=RC2, md_edge=sysm.edge)
    a.upload(ids, sysm.u)
    b = make_pool(gc, torch, n, n, lj_rc2=RC2, md_edge=sysm.edge)
    b.upload(ids, sysm.u)
    batch = host_md_batch(gc, orc, sysm, dim)
    for step in range(2):
        launches0 = a.stats()["kernel_launches"]
        a.build_md(cell, m, dim=dim)
        a.flush()
        b.submit_csr(*batch[:5], shifts=batch[5])
        b.flush()
        ra, rb = a.results(), b.results()
        assert np.array_equal(ra, rb), step
        assert np.array_equal(a.totals(ids), b.totals(ids)), step
        assert a.stats()["kernel_launches"] > launches0
    # build + one more task in the same batch: general path, same totals
    a.build_md(cell, m, dim=dim)
    a.submit_csr(np.array([gc.GC_LJ_SELF], np.uint32), np.array([0, 2], np.uint64),
                 np.array([0, 1], np.uint32), np.zeros(2, np.uint64), np.zeros(0, np.uint32))
    a.flush()
    b.submit_csr(*batch[:5], shifts=batch[5])
    b.submit_csr(np.array([gc.GC_LJ_SELF], np.uint32), np.array([0, 2], np.uint64),
                 np.array([0, 1], np.uint32), np.zeros(2, np.uint64), np.zeros(0, np.uint32))
    b.flush()
    assert np.array_equal(a.totals(ids), b.totals(ids))
    a.close()
    b.close()


def test_bad_cell_index_reported_and_pool_stays_usable(gc, orc, small_md):
    """A cell index outside the m^3 grid is an argument error of the build;
    the pool then builds and runs the valid system."""
    sysm = small_md
    n, m = sysm.n, sysm.ncell
    pool = make_pool(gc, torch, n, n, lj_rc2=RC2, md_edge=sysm.edge)
    pool.upload(np.arange(n, dtype=np.uint32), sysm.u)
    bad = sysm.cell.astype(np.int32).copy()
    bad[n // 2] = m ** 3
    with pytest.raises(gc.GcError) as e:
        pool.build_md(torch.from_numpy(bad).cuda(), m)
    assert e.value.code == gc.GC_ERR_ARG
    pool.build_md(torch.from_numpy(sysm.cell.astype(np.int32)).cuda(), m)
    pool.flush()
    start, atoms = pool.md_cells(n, m)
    s0, a0 = orc.md_cells(sysm.cell, m ** 3)
    assert np.array_equal(start, s0) and np.array_equal(atoms, a0)
    assert pool.stats()["lj_pairs_in_cutoff"] > 0
    pool.close()
