"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times: N-body at 1,048,576 Plummer particles (Section 4.1),
Lennard-Jones at 1,048,576 atoms in 42^3 cells (Section 4.2) and 200,000
uneven tasks over a 4,194,304-particle merger under a 2 GiB staging budget.
Integer work is compared in full where the oracle finishes in seconds (tree,
buckets, cells) and on seeded samples otherwise (lists, pack permutations);
forces on sampled tasks against the FP64 oracle; the rest through
properties that hold at any size (chare-table mapping, per-id totals equal
to the FP64 sums of the rows)."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import EPS2, RC2, RC2_GRID, TOL, per_task_errors, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NONE32 = 0xFFFFFFFF


@pytest.fixture(scope="module")
def gc():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    return gcharm


def pool_for(gc, id_cap, **kw):
    # the pool the benchmark creates: its own stream
    stream = torch.cuda.Stream()
    return gc.Pool(id_capacity=id_cap, pool_capacity=id_cap, eps2=EPS2,
                   stream=stream.cuda_stream, **kw), stream


def check_chare_table(pool, tg, sr):
    """First flush into an empty pool: the referenced ids take slots 0..U-1
    in ascending id order, and every entry carries its id's slot."""
    s2o, o2s, _ = pool.residency()
    ref = np.flatnonzero(s2o != NONE32)
    assert np.array_equal(s2o[ref], np.arange(ref.shape[0], dtype=np.uint32))
    assert np.array_equal(o2s[:ref.shape[0]], ref.astype(np.uint32))
    st, ss = pool.entry_slots()
    assert np.array_equal(st, s2o[tg])
    assert np.array_equal(ss, s2o[sr])
    return st, ss, ref


def check_pack_sample(pool, off, slots, sample, src):
    pt, ps = pool.pack_perm()
    perm = ps if src else pt
    for t in sample:
        a, b = int(off[t]), int(off[t + 1])
        exp = np.argsort(slots[a:b], kind="stable").astype(np.uint32)
        assert np.array_equal(perm[a:b], exp), t


def test_nbody_1m(gc, orc):
    n = 1 << 20
    x = inputs.plummer(n, inputs.SEED_BASE + 2)
    pool, stream = pool_for(gc, 2 * n + 1024)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    xd = torch.from_numpy(x).cuda()
    info = pool.build_nbody(xd, 32, 7, 10)
    g = pool.nbody_tree(n, info["n_nodes"], info["n_buckets"], info["list_entries"])
    pool.flush()
    stream.synchronize()
    tr = orc.Tree(x)
    assert info["n_nodes"] == tr.n_nodes and info["n_buckets"] == tr.n_buckets
    assert np.array_equal(g["sorted_ids"], tr.sorted_ids)
    assert np.array_equal(g["sorted_keys"], tr.sorted_keys)
    for k in ["level", "first", "count", "leaf", "size"]:
        assert np.array_equal(g[k], getattr(tr, k)), k
    assert np.array_equal(g["cell"], tr.cell)
    assert np.array_equal(g["bucket_first"], tr.bucket_first)
    assert np.array_equal(g["bucket_count"], tr.bucket_count)
    np.testing.assert_allclose(g["node_xyzm"], tr.node_table(), rtol=2e-7, atol=1e-12)
    # sampled buckets: lists bit-exact, forces within tolerance
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(tr.n_buckets, 300, replace=False))
    lo, li = tr.lists(7, 10, buckets=sample)
    to_s, tg_s = tr.bucket_targets(buckets=sample)
    goff = g["list_off"]
    for k, b in enumerate(sample):
        got = g["list_ids"][int(goff[b]):int(goff[b + 1])]
        assert np.array_equal(got, li[int(lo[k]):int(lo[k + 1])]), b
    tab = np.concatenate([x, tr.node_table()])
    ref = orc.gravity_batch(tab, to_s, tg_s, lo, li, EPS2)
    to_all, tg_all = np.zeros(tr.n_buckets + 1, np.uint64), g["sorted_ids"]
    to_all[1:] = np.cumsum(g["bucket_count"])
    assert np.array_equal(g["bucket_first"], to_all[:-1])   # buckets partition in order
    rows = pool.values()
    got = np.concatenate([rows[int(to_all[b]):int(to_all[b + 1])] for b in sample])
    errs = per_task_errors(got, ref, to_s)
    assert errs.max() <= TOL, errs.max()
    # chare table and pack permutation of the sampled lists
    st, ss, ref_ids = check_chare_table(pool, tg_all, g["list_ids"])
    assert ref_ids.shape[0] == pool.stats()["last_unique"]
    check_pack_sample(pool, goff, ss, sample, src=True)
    # per-id totals: each particle is the target of one bucket
    tot = pool.totals(tg_s)
    assert rel_l2(tot[:, :3], ref[:, :3]) <= TOL
    pool.close()


def test_md_1m(gc, orc):
    sysm = inputs.fcc_lj(64, inputs.SEED_BASE + 3, ncell=42)
    n, m = sysm.n, sysm.ncell
    pool, stream = pool_for(gc, n, lj_rc2=RC2, md_edge=sysm.edge)
    pool.upload(np.arange(n, dtype=np.uint32), sysm.u)
    info = pool.build_md(torch.from_numpy(sysm.cell.astype(np.int32)).cuda(), m)
    pool.flush()
    stream.synchronize()
    start, atoms = pool.md_cells(n, m)
    s0, a0 = orc.md_cells(sysm.cell, m ** 3)
    assert np.array_equal(start, s0) and np.array_equal(atoms, a0)
    ta, tb, td, ts = orc.md_tasks(m)
    assert info["tasks"] == len(ta) == 14 * m ** 3
    cnt = (s0[1:] - s0[:-1]).astype(np.int64)
    rows_per = cnt[ta] + np.where(ts != 0, 0, cnt[tb])
    roff = np.zeros(len(ta) + 1, np.int64)
    roff[1:] = np.cumsum(rows_per)
    rows = pool.values()
    assert rows.shape[0] == roff[-1]
    # sampled tasks against the oracle, Newton III inside each
    rng = np.random.default_rng(12)
    errs = []
    for k in rng.choice(len(ta), 2000, replace=False):
        A = a0[s0[ta[k]]:s0[ta[k] + 1]]
        B = a0[s0[tb[k]]:s0[tb[k] + 1]]
        fa, fb = orc.lj(sysm.u, A, None if ts[k] else B, bool(ts[k]), td[k], sysm.E,
                        rc2_grid=RC2_GRID)
        ref = fa if ts[k] else np.concatenate([fa, fb])
        g = rows[roff[k]:roff[k + 1]]
        errs.append(rel_l2(g[:, :3], ref[:, :3]))
        assert np.max(np.abs(g[:, :3].sum(axis=0))) <= 1e-5 * max(np.abs(g[:, :3]).sum(), 1e-30)
    assert max(errs) <= TOL, max(errs)
    # per-atom totals of sampled cells: every task touching the cell
    tot_cells = rng.choice(m ** 3, 40, replace=False)
    for c in tot_cells:
        A = a0[s0[c]:s0[c + 1]]
        ref = np.zeros((A.shape[0], 4))
        for k in np.flatnonzero((ta == c) | (tb == c)):
            Ak = a0[s0[ta[k]]:s0[ta[k] + 1]]
            Bk = a0[s0[tb[k]]:s0[tb[k] + 1]]
            fa, fb = orc.lj(sysm.u, Ak, None if ts[k] else Bk, bool(ts[k]), td[k], sysm.E,
                            rc2_grid=RC2_GRID)
            if ta[k] == c:
                ref += fa
            if not ts[k] and tb[k] == c:
                ref += fb
        tot = pool.totals(A)
        assert rel_l2(tot[:, :3], ref[:, :3]) <= TOL, c
        np.testing.assert_allclose(tot[:, 3], ref[:, 3], rtol=1e-5, atol=1e-6)
    pool.close()


def test_uneven_200k(gc, orc):
    n1, n2 = 3 << 20, 1 << 20
    n = n1 + n2
    x = inputs.merger(n1, n2, inputs.SEED_BASE + 4)
    pool, stream = pool_for(gc, 2 * n + 1024, staging_budget_bytes=2 << 30)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    pool.build_nbody(x, 32, 7, 10)
    pool.flush()
    order = pool.nbody_sorted_ids(n)
    T = 200_000
    to, tg, so, sr = inputs.uneven_tasks(n, T, inputs.SEED_BASE + 5, order=order)
    # device task arrays, alive until the flush has read them
    dev = [torch.from_numpy(a.view(t)).cuda() for a, t in
           [(np.zeros(T, np.uint32), np.int32), (to, np.int64), (tg, np.int32),
            (so, np.int64), (sr, np.int32)]]
    torch.cuda.synchronize()
    pool.reset_totals()
    pool.submit_csr_device(*dev, tg.shape[0], sr.shape[0])
    pool.flush()
    stream.synchronize()
    del dev
    st = pool.stats()
    assert st["last_waves"] > 1
    nt = (to[1:] - to[:-1]).astype(np.int64)
    ns = (so[1:] - so[:-1]).astype(np.int64)
    rows = pool.results()
    assert rows.shape[0] == tg.shape[0]
    rng = np.random.default_rng(13)
    sample = np.sort(rng.choice(T, 300, replace=False))
    # the longest task too (merged pack path)
    sample = np.unique(np.append(sample, np.argmax(ns)))
    sto = np.zeros(len(sample) + 1, np.uint64)
    sto[1:] = np.cumsum(nt[sample])
    sso = np.zeros(len(sample) + 1, np.uint64)
    sso[1:] = np.cumsum(ns[sample])
    stg = np.concatenate([tg[to[t]:to[t + 1]] for t in sample])
    ssr = np.concatenate([sr[so[t]:so[t + 1]] for t in sample])
    ref = orc.gravity_batch(x, sto, stg, sso, ssr, EPS2)
    got = np.concatenate([gc.value(rows[to[t]:to[t + 1]]) for t in sample])
    errs = per_task_errors(got, ref, sto)
    assert errs.max() <= TOL, errs.max()
    # chare-table mapping and the pack permutation of sampled lists
    st_, ss_ = pool.entry_slots()
    s2o, _, _ = pool.residency()
    assert np.array_equal(st_, s2o[tg]) and np.array_equal(ss_, s2o[sr])
    check_pack_sample(pool, so, ss_, sample, src=True)
    check_pack_sample(pool, to, st_, sample, src=False)
    # per-id totals = FP64 sums of the rows (value s - c) in admission order,
    # bit for bit (same widening, same order, same FP64 adds)
    ids = rng.choice(np.unique(tg[:: 997]), 50, replace=False)
    sel = np.isin(tg, ids)
    val = rows[sel, :4].astype(np.float64) - rows[sel, 4:].astype(np.float64)
    exp = np.zeros((n, 4))
    np.add.at(exp, tg[sel], val)
    tot = pool.totals(ids.astype(np.uint32))
    assert np.array_equal(tot, exp[ids])
    pool.close()
