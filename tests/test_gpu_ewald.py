"""GPU parity of the Ewald correction tasks (periodic gravity, the tree
code's second combined kernel, Section 4.1) against the FP64 oracle: alone,
in a batch mixed with gravity and Lennard-Jones tasks, one launch per task,
and the error path without a periodic box."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import EPS2, RC2, RC2_GRID, TOL, make_pool, per_task_errors, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 1.0


@pytest.fixture(scope="module")
def gc():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    return gcharm


def box_particles(n, seed):
    g = inputs.rng(seed)
    x = np.empty((n, 4), np.float32)
    x[:, :3] = g.uniform(0.0, L, size=(n, 3))
    x[:, 3] = g.uniform(0.5, 1.5, size=n) / n
    return x


def ewald_tasks(n, n_tasks, seed):
    g = inputs.rng(seed)
    nt = g.integers(1, 33, n_tasks)
    ns = g.integers(1, 9, n_tasks)
    to = np.concatenate([[0], np.cumsum(nt)]).astype(np.uint64)
    so = np.concatenate([[0], np.cumsum(ns)]).astype(np.uint64)
    tg = g.integers(0, n, int(to[-1])).astype(np.uint32)
    sr = g.integers(0, n, int(so[-1])).astype(np.uint32)
    sr[0] = tg[0]                                  # a target that is its own source (r = 0)
    return to, tg, so, sr


def oracle_rows(orc, x, to, tg, so, sr):
    return np.concatenate([orc.ewald(x, tg[to[t]:to[t + 1]], sr[so[t]:so[t + 1]], L)
                           for t in range(len(to) - 1)])


def test_ewald_batch_vs_oracle(gc, orc):
    n = 3000
    x = box_particles(n, 81)
    to, tg, so, sr = ewald_tasks(n, 60, 82)
    pool = make_pool(gc, torch, n, n, ewald_box=L)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    kinds = np.full(len(to) - 1, gc.GC_EWALD, np.uint32)
    b = pool.submit_csr(kinds, to, tg, so, sr)
    pool.flush()
    pool.wait(b)
    got = pool.values()
    ref = oracle_rows(orc, x, to, tg, so, sr)
    errs = per_task_errors(got, ref, to)
    assert errs.max() <= TOL, errs.max()
    # potentials too (same tolerance on the phi column, per task)
    for t in range(len(to) - 1):
        a, c = int(to[t]), int(to[t + 1])
        assert rel_l2(got[a:c, 3], ref[a:c, 3]) <= TOL
    assert pool.stats()["interactions"] == int(((to[1:] - to[:-1]) * (so[1:] - so[:-1])).sum())
    # one launch per task: the same kernel, the same rows
    b = pool.submit_csr(kinds, to, tg, so, sr)
    pool.flush_per_task()
    pool.wait(b)
    assert np.array_equal(pool.values(), got)
    pool.close()


def test_ewald_in_a_mixed_batch(gc, orc):
    # gravity, LJ and Ewald tasks in one combined batch (one flush)
    n = 2048
    x = box_particles(n, 83)
    sysm = inputs.fcc_lj(8, inputs.SEED_BASE + 3, ncell=5)       # 2048 LJ atoms
    ids_md = np.arange(n, 2 * n, dtype=np.uint32)
    pool = make_pool(gc, torch, 2 * n, 2 * n, ewald_box=L, lj_rc2=RC2, md_edge=sysm.edge)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    pool.upload(ids_md, sysm.u)
    to_g, tg_g, so_g, sr_g = inputs.uneven_tasks(n, 20, 84, (1, 32), (1, 500))
    to_e, tg_e, so_e, sr_e = ewald_tasks(n, 20, 85)
    start, atoms = orc.md_cells(sysm.cell, sysm.ncell ** 3)
    ta, tb, td, ts = orc.md_tasks(sysm.ncell)
    pick = [k for k in range(len(ta)) if not ts[k]][:10]
    A = [atoms[start[ta[k]]:start[ta[k] + 1]] for k in pick]
    B = [atoms[start[tb[k]]:start[tb[k] + 1]] for k in pick]
    tasks = []
    for t in range(20):
        tasks.append(dict(kind=gc.GC_GRAVITY, targets=tg_g[to_g[t]:to_g[t + 1]],
                          sources=sr_g[so_g[t]:so_g[t + 1]]))
        tasks.append(dict(kind=gc.GC_EWALD, targets=tg_e[to_e[t]:to_e[t + 1]],
                          sources=sr_e[so_e[t]:so_e[t + 1]]))
        if t < len(pick):
            tasks.append(dict(kind=gc.GC_LJ_PAIR, targets=A[t] + n, sources=B[t] + n,
                              shift=tuple(int(v) for v in td[pick[t]])))
    b = pool.submit_tasks(tasks)
    pool.flush()
    pool.wait(b)
    got = pool.values()
    row = 0
    for t, d in enumerate(tasks):
        tg = np.asarray(d["targets"], np.uint32)
        sr = np.asarray(d["sources"], np.uint32)
        if d["kind"] == gc.GC_GRAVITY:
            ref = orc.gravity(x, tg, sr, EPS2)
        elif d["kind"] == gc.GC_EWALD:
            ref = orc.ewald(x, tg, sr, L)
        else:
            u = np.concatenate([x, sysm.u])          # ids n.. are the LJ atoms
            fa, fb = orc.lj(u, tg, sr, False, d["shift"], sysm.E, rc2_grid=RC2_GRID)
            ref = np.concatenate([fa, fb])
        g = got[row:row + len(ref)]
        row += len(ref)
        assert rel_l2(g[:, :3], ref[:, :3]) <= TOL, (t, d["kind"])
    assert row == got.shape[0]
    pool.close()


def test_ewald_needs_a_box(gc):
    pool = make_pool(gc, torch, 16, 16)
    pool.upload(np.arange(16, dtype=np.uint32), box_particles(16, 86))
    with pytest.raises(gc.GcError) as e:
        pool.submit_csr(np.array([gc.GC_EWALD], np.uint32), np.array([0, 2], np.uint64),
                        np.array([0, 1], np.uint32), np.array([0, 1], np.uint64),
                        np.array([2], np.uint32))
    assert e.value.code == gc.GC_ERR_ARG
    pool.close()
