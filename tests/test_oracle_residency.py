"""Pins for the oracle's chare table (residency), pack permutation and
cross-task reduction (Section 3.2: reuse of resident data through the chare
table; data indices kept sorted by binary-search insertion, Fig. 1d)."""
import numpy as np

from paper_2008_05712_gb300 import inputs

NONE = 0xFFFFFFFF


def test_hand_trace(orc):
    # capacity 3, ids < 8
    R = orc.Residency(8, 3)
    rc, r = R.flush([5, 2, 5], epoch=1)
    assert rc == 0 and r["misses"] == 2 and r["hits"] == 0
    assert list(r["slots"]) == [1, 0, 1]          # id 2 -> slot 0, id 5 -> slot 1
    assert list(r["reuse"]) == [1, 2]
    rc, r = R.flush([7, 1], epoch=2)
    # misses 1, 7; one free slot (2); evict the oldest unreferenced entry with
    # the lowest slot: id 2 (slot 0, last use 1); then id 1 -> 0, id 7 -> 2
    assert rc == 0 and r["evictions"] == 1 and list(r["evicted"]) == [2]
    assert list(r["slots"]) == [2, 0]
    rc, r = R.flush([5, 1], epoch=3)
    assert rc == 0 and r["hits"] == 2 and r["misses"] == 0 and list(r["slots"]) == [1, 0]
    rc, r = R.flush([2, 3], epoch=4)
    # candidates: id 7 (slot 2, last 2) is older than 5 and 1 (last 3):
    # evict id 7 first, then (last 3) the lower slot: id 1 (slot 0)
    assert rc == 0 and sorted(r["evicted"].tolist()) == [1, 7]
    assert list(r["slots"]) == [0, 2]
    # a batch larger than the pool cannot be placed; the state is untouched
    before = (R.slot_of_id.copy(), R.id_of_slot.copy())
    rc, r = R.flush([0, 1, 4, 6], epoch=5)
    assert rc == -3
    assert np.array_equal(before[0], R.slot_of_id) and np.array_equal(before[1], R.id_of_slot)


def check_invariants(R, before, entry, epoch, r):
    slot_b, idslot_b, last_b = before
    U = np.unique(entry)
    assert np.array_equal(r["uniq"], U)
    _, cnt = np.unique(entry, return_counts=True)
    assert np.array_equal(r["reuse"], cnt)
    resident_b = slot_b[U] != NONE
    assert r["hits"] == int(resident_b.sum()) and r["misses"] == int((~resident_b).sum())
    # hits keep their slot
    assert np.array_equal(R.slot_of_id[U[resident_b]], slot_b[U[resident_b]])
    # the two maps are inverse
    res = np.nonzero(R.slot_of_id != NONE)[0]
    assert np.array_equal(R.id_of_slot[R.slot_of_id[res]], res)
    assert (R.id_of_slot != NONE).sum() == len(res)
    # eviction count and choice: oldest (last_use, slot) among unreferenced
    free_b = int((idslot_b == NONE).sum())
    need = max(0, r["misses"] - free_b)
    assert r["evictions"] == need
    if need:
        cand = [s for s in range(len(idslot_b)) if idslot_b[s] != NONE and idslot_b[s] not in set(U)]
        order = sorted(cand, key=lambda s: (int(last_b[s]), s))
        assert sorted(r["evicted"].tolist()) == sorted(int(idslot_b[s]) for s in order[:need])
    # misses (ascending id) take the lowest free slots in ascending order
    miss = U[~resident_b]
    ms = R.slot_of_id[miss]
    assert np.all(np.diff(ms.astype(np.int64)) > 0)
    free_after_evict = np.nonzero((idslot_b == NONE) | np.isin(idslot_b, r["evicted"]))[0]
    assert np.array_equal(ms, free_after_evict[:len(miss)])
    assert np.all(R.last_use[R.slot_of_id[U]] == epoch)
    assert np.array_equal(r["slots"], R.slot_of_id[entry])


def test_policy_invariants_random(orc):
    R = orc.Residency(1000, 200)
    for k, batch in enumerate(inputs.random_id_batches(1000, 30, 150, seed=9, hot=0.6)):
        before = (R.slot_of_id.copy(), R.id_of_slot.copy(), R.last_use.copy())
        rc, r = R.flush(batch, epoch=k + 1)
        if rc == -3:
            assert len(np.unique(batch)) > 200
            continue
        assert rc == 0
        check_invariants(R, before, batch, k + 1, r)


def test_pack_perm_is_stable_sort(orc):
    g = inputs.rng(4)
    for n in [0, 1, 2, 7, 64, 1000]:
        s = g.integers(0, 50, n).astype(np.uint32)     # many ties
        assert np.array_equal(orc.pack_perm(s), np.argsort(s, kind="stable"))
    # hand example
    assert orc.pack_perm(np.array([9, 3, 9, 1], np.uint32)).tolist() == [3, 1, 0, 2]
    off = np.array([0, 3, 3, 8], np.uint64)
    s = np.array([5, 1, 5, 4, 4, 0, 9, 4], np.uint32)
    assert orc.pack_perm_batch(off, s).tolist() == [1, 0, 2, 2, 0, 1, 4, 3]


def test_reduce_order_and_stride(orc):
    """Cross-task reduction (Section 2.2: the results of the combined kernel
    go back to each chare): per id, an FP64 sum taken in admission order.

    Hand-worked values.  In binary64 the spacing of numbers near 1e16 is 2, so
    1e16 + 1 is a tie that rounds to the even neighbour 1e16: admitted as
    (1e16, 1, -1e16) the total is exactly 0, admitted as (1e16, -1e16, 1) it
    is exactly 1.  A reversed or reassociated order, an FP32 accumulator or
    a compensated sum would each give the other value for one of the two ids.
    """
    big = 1e16
    id_cap = 9
    # rows in admission order: (id, 4 components)
    rows = [
        (3, [big, 0.5, 0.0, -2.0]),
        (8, [big, 1.0, 0.0, 0.0]),       # the top id of the range
        (3, [1.0, 0.25, 0.0, -2.0]),
        (8, [-big, 2.0, 0.0, 0.0]),
        (3, [-big, 0.125, 7.0, -2.0]),
        (8, [1.0, 4.0, 0.0, 3.0]),
        (0, [0.0, 0.0, -1.5, 0.0]),
    ]
    ids = np.array([r[0] for r in rows], np.uint32)
    c = np.array([r[1] for r in rows], np.float64)
    tot = orc.reduce(ids, c, id_cap)
    assert tot.shape == (id_cap, 4)
    assert tot[3].tolist() == [0.0, 0.875, 7.0, -6.0]
    assert tot[8].tolist() == [1.0, 7.0, 0.0, 3.0]
    assert tot[0].tolist() == [0.0, 0.0, -1.5, 0.0]
    for i in (1, 2, 4, 5, 6, 7):                 # never referenced
        assert tot[i].tolist() == [0.0, 0.0, 0.0, 0.0]
    # the same rows admitted in another order (rows 2 <-> 4 and 3 <-> 5, so
    # id 3 sees 1e16, -1e16, 1 and id 8 sees 1e16, 1, -1e16) swap the two
    # outcomes; the other components are exact in any order
    order = [0, 1, 4, 5, 2, 3, 6]
    tot_r = orc.reduce(ids[order].copy(), c[order].copy(), id_cap)
    assert tot_r[3].tolist() == [1.0, 0.875, 7.0, -6.0]
    assert tot_r[8].tolist() == [0.0, 7.0, 0.0, 3.0]
    # no rows: all zero
    assert not orc.reduce(np.zeros(0, np.uint32), np.zeros((0, 4)), 4).any()


def test_reduce_three_tasks_one_id(orc):
    """One id referenced by three tasks, each contributing distinct powers of
    two per component (exact in FP64), next to a neighbour id: the totals
    show each component landing in its own column and no row leaking into
    the neighbouring id."""
    ids = np.array([5, 4, 5, 6, 5], np.uint32)
    c = np.array([[1, 2, 4, 8],
                  [16, 32, 64, 128],
                  [256, 512, 1024, 2048],
                  [4096, 8192, 16384, 32768],
                  [65536, 131072, 262144, 524288]], np.float64)
    tot = orc.reduce(ids, c, 7)
    assert tot[5].tolist() == [65793.0, 131586.0, 263172.0, 526344.0]
    assert tot[4].tolist() == [16.0, 32.0, 64.0, 128.0]
    assert tot[6].tolist() == [4096.0, 8192.0, 16384.0, 32768.0]
    assert not tot[[0, 1, 2, 3]].any()
