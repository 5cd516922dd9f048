"""Pins for the oracle's octree, buckets and interaction-list walk
(Section 4.1: buckets of particles sharing one interaction list of tree
nodes and particles from a Barnes-Hut tree walk)."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs


def test_morton_hand_values(orc):
    # Coordinates on an exact grid: lo = 0, extent 1 -> L = 1, q = x * 2^21.
    pts = np.array([[0, 0, 0, 1],
                    [2 ** -21, 0, 0, 1],
                    [0, 2 ** -21, 0, 1],
                    [0, 0, 2 ** -21, 1],
                    [3 * 2 ** -21, 0, 0, 1],
                    [1.0, 1.0, 1.0, 1]], dtype=np.float32)
    keys, q3, lo, L = orc.morton_keys(pts)
    assert L == 1.0 and np.all(lo == 0)
    assert keys[0] == 0
    assert keys[1] == 1 and keys[2] == 2 and keys[3] == 4
    assert keys[4] == 1 + 8
    # x = 1.0 maps to 2^21, clamped to 2^21 - 1 on every axis -> all 63 bits
    assert list(q3[5]) == [2 ** 21 - 1] * 3
    assert keys[5] == 2 ** 63 - 1


def test_power_of_two_extent(orc):
    pts = np.array([[-1, 0, 0, 1], [2, 0.5, 0, 1]], dtype=np.float32)
    _, q3, lo, L = orc.morton_keys(pts)
    assert L == 4.0 and lo[0] == -1.0
    # x = 2: (2 - (-1)) * 2^21 / 4 = 1572864
    assert q3[1, 0] == 1572864 and q3[1, 1] == 2 ** 18


def test_cube_corners_tree(orc):
    # 8 particles at the corners of a cube, bucket_max = 1: root + 8 leaves in
    # octant order (bit0 = x, bit1 = y, bit2 = z), preorder ids 0..8
    pts = []
    for o in range(8):
        pts.append([float(o & 1), float((o >> 1) & 1), float((o >> 2) & 1), 1.0 + o])
    tr = orc.Tree(np.array(pts, np.float32), bucket_max=1)
    assert tr.n_nodes == 9 and tr.n_buckets == 8
    assert tr.leaf[0] == 0 and tr.size[0] == 9 and tr.count[0] == 8
    assert list(tr.child[0]) == list(range(1, 9))
    for o in range(8):
        k = 1 + o
        assert tr.level[k] == 1 and tr.leaf[k] == 1 and tr.count[k] == 1
        assert list(tr.cell[k]) == [o & 1, (o >> 1) & 1, (o >> 2) & 1]
        assert tr.sorted_ids[tr.first[k]] == o
    assert tr.mono[0, 0] == pytest.approx(sum(1.0 + o for o in range(8)), rel=1e-15)


def test_two_clusters_hand_tree(orc):
    # 3 particles near the origin corner, 2 in the far corner, bucket_max 2:
    # root splits; octant 0 holds 3 > 2 particles and splits again.
    pts = np.array([[0.0, 0.0, 0.0, 1],
                    [0.3, 0.0, 0.0, 1],
                    [0.0, 0.3, 0.0, 1],
                    [0.9, 0.9, 0.9, 1],
                    [1.0, 1.0, 1.0, 1]], np.float32)
    tr = orc.Tree(pts, bucket_max=2)
    # preorder: 0 root, 1 octant-0 cell (3 particles), its children
    # (sub-octants 0 (id 0), 1 (id 1), 2 (id 2)), then octant 7 (ids 3, 4)
    assert tr.n_nodes == 6
    assert list(tr.level) == [0, 1, 2, 2, 2, 1]
    assert list(tr.count) == [5, 3, 1, 1, 1, 2]
    assert list(tr.leaf) == [0, 0, 1, 1, 1, 1]
    assert list(tr.size) == [6, 4, 1, 1, 1, 1]
    assert list(tr.sorted_ids) == [0, 1, 2, 3, 4]
    assert tr.n_buckets == 4
    assert list(tr.bucket_count) == [1, 1, 1, 2]


@pytest.fixture(scope="module")
def c1(orc):
    x = inputs.plummer(4096, inputs.SEED_BASE + 1)
    return x, orc.Tree(x)


def test_buckets_partition(c1):
    x, tr = c1
    n = x.shape[0]
    assert sorted(tr.sorted_ids.tolist()) == list(range(n))
    assert np.all(np.diff(tr.sorted_keys.astype(np.float64)) >= 0)
    b_end = tr.bucket_first.astype(np.int64) + tr.bucket_count
    assert tr.bucket_first[0] == 0 and b_end[-1] == n
    assert np.all(tr.bucket_first[1:] == b_end[:-1])
    assert tr.bucket_count.max() <= 32 and tr.bucket_count.min() >= 1
    # buckets are leaves: a node of count <= 32 (or at the finest level)
    assert np.all(tr.leaf[tr.bucket_node] == 1)


def test_node_invariants(c1):
    x, tr = c1
    m = x[:, 3].astype(np.float64)
    srt = tr.sorted_ids
    for k in range(tr.n_nodes):
        f, c = int(tr.first[k]), int(tr.count[k])
        assert tr.mono[k, 0] == pytest.approx(m[srt[f:f + c]].sum(), rel=1e-14)
        if not tr.leaf[k]:
            kids = [int(v) for v in tr.child[k] if v != 0xFFFFFFFF]
            assert sum(int(tr.count[q]) for q in kids) == c
            assert 1 + sum(int(tr.size[q]) for q in kids) == tr.size[k]
            assert kids[0] == k + 1
            assert c > 32


def test_theta_zero_is_direct_sum(c1, orc):
    x, tr = c1
    off, ids = tr.lists(0, 1, buckets=range(0, tr.n_buckets, 37))
    lens = np.diff(off.astype(np.int64))
    assert np.all(lens == x.shape[0])
    for t in range(len(lens)):
        seg = ids[off[t]:off[t + 1]]
        assert np.array_equal(np.sort(seg), np.arange(x.shape[0]))


def test_list_mass_covers_total(c1):
    # every list (nodes + particles) covers each particle exactly once, so
    # the masses of its entries sum to the total mass
    x, tr = c1
    n = x.shape[0]
    m_node = tr.mono[:, 0]
    m_part = x[:, 3].astype(np.float64)
    off, ids = tr.lists(7, 10)
    total = m_part.sum()
    for t in range(len(off) - 1):
        seg = ids[off[t]:off[t + 1]].astype(np.int64)
        mass = np.where(seg < n, m_part[np.minimum(seg, n - 1)],
                        m_node[np.maximum(seg - n, 0)]).sum()
        assert mass == pytest.approx(total, rel=1e-13), t


def test_theta_large_is_minimal_list(c1):
    # with a huge opening angle every node that does not contain the bucket
    # is accepted: the list is the siblings of each ancestor of the bucket's
    # leaf (in root-to-leaf order) plus the leaf's particles
    x, tr = c1
    n = x.shape[0]
    parent = np.full(tr.n_nodes, -1)
    for k in range(tr.n_nodes):
        for c in tr.child[k]:
            if c != 0xFFFFFFFF:
                parent[c] = k
    for b in range(0, tr.n_buckets, 11):
        leaf = int(tr.bucket_node[b])
        path = [leaf]
        while parent[path[-1]] >= 0:
            path.append(int(parent[path[-1]]))
        path = path[::-1]

        def expect_from(depth):
            p = path[depth]
            out = []
            for c in tr.child[p]:
                if c == 0xFFFFFFFF:
                    continue
                if c == path[depth + 1]:
                    if c == leaf:
                        f, cnt = int(tr.first[c]), int(tr.count[c])
                        out.extend(tr.sorted_ids[f:f + cnt].tolist())
                    else:
                        out.extend(expect_from(depth + 1))
                else:
                    out.append(n + int(c))
            return out

        expect = expect_from(0)
        got = tr.walk(b, 255, 1)
        # the leaf's particles sit where the leaf is in octant order
        assert got.tolist() == expect, b


def test_bh_error_vs_direct(c1, orc):
    # theta = 0.7 lists reproduce the direct sum to the accuracy expected of
    # a monopole expansion (well below 1 %), theta = 0 is exact
    x, tr = c1
    tab = np.concatenate([x, tr.node_table()])
    bs = list(range(0, tr.n_buckets, 5))
    to, tg = tr.bucket_targets(bs)
    off7, ids7 = tr.lists(7, 10, bs)
    off0, ids0 = tr.lists(0, 1, bs)
    a7 = orc.gravity_batch(tab, to, tg, off7, ids7, np.float32(1e-4))
    a0 = orc.gravity_batch(tab, to, tg, off0, ids0, np.float32(1e-4))
    ad = orc.gravity(x, tg, np.arange(x.shape[0], dtype=np.uint32), np.float32(1e-4))
    np.testing.assert_allclose(a0, ad, rtol=1e-10, atol=1e-12)
    e = np.linalg.norm(a7[:, :3] - ad[:, :3]) / np.linalg.norm(ad[:, :3])
    assert e < 1e-2
