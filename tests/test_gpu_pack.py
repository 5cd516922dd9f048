"""GPU parity of the sorted pack (Section 3.2, Fig. 1d) on lists built to
stress the sort: every size-class boundary (32/33, 1024/1025, 2048/2049,
4096/4097, 16384/16385 and a list merged from three sorted chunks),
lists of one repeated id (no radix pass needed), lists with heavy
duplication (stability decides the order), lists spanning the whole slot
range and lists confined to a narrow one, lists already in order, lists in
order but for one low slot at the end, and lists shaped like the N-body
interaction lists (an ascending tail of high slots interleaved with short
runs of random low ones).  The pack permutation must equal a
stable argsort of the entry slots, bit for bit, and the staged forces must
match the FP64 oracle."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import EPS2, TOL, make_pool, per_task_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    return gcharm


def adversarial_lists(n_ids, seed):
    rng = np.random.default_rng(seed)
    lists = []
    for size in (31, 32, 33, 34, 500, 1023, 1024, 1025, 1500, 2047, 2048, 2049, 3000,
                 4095, 4096, 4097, 10000, 16384, 16385, 40000):
        lists.append(rng.integers(0, n_ids, size))                     # full range
        lists.append(np.full(size, rng.integers(0, n_ids)))            # one id
        lists.append(rng.integers(0, 7, size) * 997 % n_ids)           # 7 distinct ids
        base = int(rng.integers(0, n_ids - 70))
        lists.append(base + rng.integers(0, 64, size))                 # narrow range
        lists.append(np.sort(rng.integers(0, n_ids, size))[::-1])      # descending
        lists.append(tree_like(rng, n_ids, size))                      # ordered tail
        asc = np.sort(rng.integers(1, n_ids, size))
        lists.append(asc.copy())                                       # in order already
        asc[-1] = 0
        lists.append(asc)                                              # one low slot last
    return [a.astype(np.uint32) for a in lists]


def tree_like(rng, n_ids, size):
    """The shape of an N-body interaction list: about two thirds ascending
    high ids (tree nodes in depth-first order) interleaved with runs of up
    to 9 random lower ids (the particles of opened leaves)."""
    cut = int(0.9 * n_ids)
    n_hi = size - size // 3
    hi = np.sort(rng.integers(cut, n_ids, n_hi))
    lo = rng.integers(0, cut, size - n_hi)
    out, i, j = [], 0, 0
    while i < len(hi) or j < len(lo):
        if j < len(lo) and (i == len(hi) or rng.random() < 0.1):
            k = min(len(lo), j + int(rng.integers(1, 10)))
            out.extend(lo[j:k])
            j = k
        else:
            out.append(hi[i])
            i += 1
    return np.array(out)


def csr(lists):
    off = np.zeros(len(lists) + 1, np.uint64)
    off[1:] = np.cumsum([len(a) for a in lists])
    return off, np.concatenate(lists)


@pytest.mark.parametrize("warm", [False, True])
def test_pack_permutation_adversarial(gc, orc, warm):
    """warm: a first batch references every id, so ids take slots 0..N-1 and
    the lists below span a 20-bit slot range; otherwise only the referenced
    ids take slots (a 16-bit range)."""
    n = 1 << 20
    x = inputs.plummer(n, 91)
    srcs = adversarial_lists(n, 92)
    rng = np.random.default_rng(93)
    # target lists cycle through the same shapes, kept distinct within a list
    tgts = [rng.choice(n, min(len(s), 2500) if len(s) <= 3000 else 48, replace=False)
            .astype(np.uint32) for s in srcs]
    to, tg = csr(tgts)
    so, sr = csr(srcs)
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    if warm:
        b = pool.submit_csr(np.zeros(1, np.uint32), np.array([0, n], np.uint64),
                            np.arange(n, dtype=np.uint32), np.array([0, 1], np.uint64),
                            np.zeros(1, np.uint32))
        pool.flush()
        pool.wait(b)
    b = pool.submit_csr(np.zeros(len(srcs), np.uint32), to, tg, so, sr)
    pool.flush()
    pool.wait(b)
    st, ss = pool.entry_slots()
    if warm:
        assert np.array_equal(ss, sr)          # slot = id after the warm batch
    pt, ps = pool.pack_perm()
    assert np.array_equal(ps, orc.pack_perm_batch(so, ss))
    assert np.array_equal(pt, orc.pack_perm_batch(to, st))
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    errs = per_task_errors(pool.values(), ref, to)
    assert errs.max() <= TOL, errs.max()
    pool.close()


def test_pack_permutation_small_lists(gc, orc):
    """Tasks whose two lists both hold at most 16 entries are sorted one list
    per half-warp; the others one list per warp.  Every combination of the
    sizes around those limits, with repeated ids, against the oracle."""
    n = 5000
    x = inputs.plummer(n, 94)
    rng = np.random.default_rng(95)
    sizes = [0, 1, 2, 7, 15, 16, 17, 31, 32]
    tgts, srcs = [], []
    for a_ in sizes:
        for b_ in sizes:
            if a_ == 0:
                continue                      # a task has at least one target
            tgts.append(rng.choice(n, a_, replace=False).astype(np.uint32))
            srcs.append(rng.integers(0, 40, b_).astype(np.uint32) * 97 % n)
    to, tg = csr(tgts)
    so, sr = csr([s.astype(np.uint32) for s in srcs])
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    b = pool.submit_csr(np.zeros(len(tgts), np.uint32), to, tg, so, sr)
    pool.flush()
    pool.wait(b)
    st, ss = pool.entry_slots()
    pt, ps = pool.pack_perm()
    assert np.array_equal(pt, orc.pack_perm_batch(to, st))
    assert np.array_equal(ps, orc.pack_perm_batch(so, ss))
    ref = orc.gravity_batch(x, to, tg, so, sr, EPS2)
    errs = per_task_errors(pool.values(), ref, to)
    assert errs.max() <= TOL, errs.max()
    pool.close()
