"""Tree rebuilds seeded by the previous step's Morton order (Section 4.1:
the tree is rebuilt at every step of the integration).

The seeded build keeps a sorted subsequence of the previous order in place
and places the particles that moved out of it next to their successors in
it.  Its order -- and so every node, bucket and list -- must equal the
oracle's from-scratch build, bit for bit, after every one of ten drift
steps.  Previous orders that help nothing (relabelled, reversed or rotated
particles) crowd many movers into one place, and the build sorts all keys
instead; coincident particles (equal keys) stay in id order either way."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import make_pool

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    return gcharm


def _check_tree(pool, info, x, orc, bucket=32, theta=(7, 10), lists=True):
    n = x.shape[0]
    g = pool.nbody_tree(n, info["n_nodes"], info["n_buckets"], info["list_entries"])
    tr = orc.Tree(x, bucket_max=bucket)
    assert np.array_equal(g["sorted_ids"], tr.sorted_ids)
    assert np.array_equal(g["sorted_keys"], tr.sorted_keys)
    assert info["n_nodes"] == tr.n_nodes and info["n_buckets"] == tr.n_buckets
    for k in ["level", "first", "count", "leaf", "size"]:
        assert np.array_equal(g[k], getattr(tr, k)), k
    assert np.array_equal(g["cell"], tr.cell)
    assert np.array_equal(g["bucket_first"], tr.bucket_first)
    assert np.array_equal(g["bucket_count"], tr.bucket_count)
    if lists:
        off, ids = tr.lists(*theta)
        assert np.array_equal(g["list_off"], off)
        assert np.array_equal(g["list_ids"], ids)
    np.testing.assert_allclose(g["node_xyzm"], tr.node_table(), rtol=2e-7, atol=1e-12)
    return tr


def _step(pool, x, bucket=32, theta=(7, 10)):
    n = x.shape[0]
    pool.upload(np.arange(n, dtype=np.uint32), x)
    info = pool.build_nbody(torch.from_numpy(x).cuda(), bucket, *theta)
    return info


@pytest.mark.parametrize("n", [65536, 30001])
def test_seeded_tree_bit_exact_over_ten_drift_steps(gc, orc, n):
    x = inputs.plummer(n, inputs.SEED_BASE + 7)
    pool = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
    resorted = []
    for step in range(11):
        if step:
            x = inputs.drift(x, inputs.SEED_BASE + 100 + step)
        info = _step(pool, x)
        _check_tree(pool, info, x, orc, lists=(step % 5 == 0))
        pool.flush()
        pool.wait(0)
        resorted.append(info["resorted"])
    st = pool.nbody_stats()
    assert st["builds"] == 11 and st["seeded_builds"] == 10
    assert resorted[0] == n                      # the first build sorts everything
    assert max(resorted[1:]) < n // 4            # a 1e-3 drift moves few particles
    assert st["timed_builds"] == 11 and st["tree_ms_sum"] > st["order_ms_sum"] > 0
    pool.close()


def test_full_and_seeded_orders_agree(gc, orc):
    n = 20000
    x = inputs.plummer(n, inputs.SEED_BASE + 8)
    pf = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
    pf.set_order(gc.GC_ORDER_FULL)
    ps = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
    for step in range(4):
        if step:
            x = inputs.drift(x, inputs.SEED_BASE + 200 + step, sigma=1e-2)
        a, b = _step(pf, x), _step(ps, x)
        assert a["resorted"] == n
        ga = pf.nbody_tree(n, a["n_nodes"], a["n_buckets"], a["list_entries"])
        gb = ps.nbody_tree(n, b["n_nodes"], b["n_buckets"], b["list_entries"])
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), (step, k)
        pf.flush()
        ps.flush()
        pf.wait(0)
        ps.wait(0)
    assert pf.nbody_stats()["seeded_builds"] == 0
    assert ps.nbody_stats()["seeded_builds"] == 3
    with pytest.raises(gc.GcError) as e:
        ps.set_order(7)
    assert e.value.code == gc.GC_ERR_ARG
    pf.close()
    ps.close()


def _relabel(x, perm_sorted, how, rng):
    """Positions whose previous sorted order, applied to them, gives a
    reversed, rotated or random sequence of the same keys."""
    n = x.shape[0]
    y = np.empty_like(x)
    if how == "reversed":
        y[perm_sorted] = x[perm_sorted[::-1]]
    elif how == "rotated":
        y[perm_sorted] = x[np.roll(perm_sorted, -(n // 3))]
    else:
        y = x[rng.permutation(n)]
    return y


@pytest.mark.parametrize("how", ["reversed", "rotated", "random"])
def test_seeded_order_under_unhelpful_previous_orders(gc, orc, how):
    # reversed and random: nearly every particle is a mover.  Rotated: one
    # cliff; the tiles after it fall below the kept maximum, and the tile
    # holding the cliff (one or two particles dropped per round) gives up
    # after its round limit.  Each crowds thousands of movers before one
    # kept particle: the build falls back to the full sort
    n = 9000
    rng = np.random.default_rng(inputs.SEED_BASE + 9)
    x = inputs.plummer(n, inputs.SEED_BASE + 9)
    pool = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
    info = _step(pool, x)
    tr = _check_tree(pool, info, x, orc, lists=False)
    pool.flush()
    pool.wait(0)
    y = _relabel(x, tr.sorted_ids, how, rng)
    info = _step(pool, y)
    _check_tree(pool, info, y, orc)
    assert info["resorted"] == n
    assert pool.nbody_stats()["seeded_builds"] == 0
    # the next small step is seeded again
    z = inputs.drift(y, inputs.SEED_BASE + 19)
    pool.flush()
    pool.wait(0)
    info = _step(pool, z)
    _check_tree(pool, info, z, orc, lists=False)
    assert info["resorted"] < n // 4
    assert pool.nbody_stats()["seeded_builds"] == 1
    pool.close()


def test_seeded_order_with_coincident_particles(gc, orc):
    # three particles at every position: equal keys, ordered by id
    base = inputs.plummer(3000, inputs.SEED_BASE + 10)
    x = np.repeat(base, 3, axis=0)
    n = x.shape[0]
    rng = np.random.default_rng(inputs.SEED_BASE + 10)
    pool = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
    for step in range(5):
        if step == 2:
            x = x[rng.permutation(n)]
        elif step:   # drift each position once: its three particles stay together
            u, inv = np.unique(x, axis=0, return_inverse=True)
            x = inputs.drift(u, inputs.SEED_BASE + 300 + step)[inv.ravel()]
        info = _step(pool, x)
        _check_tree(pool, info, x, orc, lists=False)
        pool.flush()
        pool.wait(0)
    # steps 1, 3 and 4 seeded; the relabelling (step 2) sorts afresh
    assert pool.nbody_stats()["seeded_builds"] == 3
    pool.close()


def test_seeded_order_after_a_size_change_sorts_afresh(gc, orc):
    pool = make_pool(gc, torch, 3 * 6000 + 64, 3 * 6000 + 64)
    for n in (5000, 6000, 6000, 1, 1):
        x = inputs.plummer(n, inputs.SEED_BASE + n)
        info = _step(pool, x)
        _check_tree(pool, info, x, orc, lists=False)
        pool.flush()
        pool.wait(0)
    st = pool.nbody_stats()
    assert st["builds"] == 5 and st["seeded_builds"] == 2
    pool.close()


def test_morton_keys_at_fp64_rounding_edges(gc, orc):
    # The keys quantise (x - lo) 2^21 / L as the FP64 expression does; the
    # kernels compute it in FP32 where that is provably the same and fall
    # back to FP64 for coordinates below 2^-(sh+6) in magnitude.  x: lo =
    # -64, L = 128 (sh = 14), with -2^-60, where the FP64 subtraction rounds
    # 64 - 2^-60 up to the grid line 64; y: a large offset (1e6) and values
    # one ulp below grid lines; z: zeros, signed zeros and subnormals.
    rng = np.random.default_rng(inputs.SEED_BASE + 11)
    xs = [-64.0, 63.9, -2.0**-60, 2.0**-60, -2.0**-20, -2.0**-21, 2.0**-20, 0.0, -0.0,
          -1e-30, 1e-45, -1e-45, 32.0, np.nextafter(np.float32(32.0), np.float32(-1)),
          np.nextafter(np.float32(-32.0), np.float32(-100))]
    ys = [1e6, 1e6 + 0.0625, 1e6 + 1.0, np.nextafter(np.float32(1e6 + 8), np.float32(0)), 1e6 + 8]
    zs = [0.0, -0.0, 2.0**-149, -2.0**-149, 2.0**-126, -1.0, 1.0, 0.5, -0.5]
    n = 3000
    x = np.empty((n, 4), np.float32)
    x[:, 0] = rng.choice(np.array(xs, np.float32), n)
    x[:, 1] = rng.choice(np.array(ys, np.float32), n)
    x[:, 2] = rng.choice(np.array(zs, np.float32), n)
    x[:, 3] = 1.0 / n
    x[0, :3] = (-64.0, 1e6, -1.0)          # the minima and the extents
    x[1, :3] = (63.9, 1e6 + 8, 1.0)
    for mode in (gc.GC_ORDER_FULL, gc.GC_ORDER_SEEDED):
        pool = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
        pool.set_order(mode)
        for step in range(3):   # the seeded pool reorders from its own order
            y = x.copy()
            y[:, :3] = x[rng.permutation(n), :3] if step == 2 else x[:, :3]
            info = _step(pool, y)
            g = pool.nbody_tree(n, info["n_nodes"], info["n_buckets"], info["list_entries"])
            tr = orc.Tree(y)
            assert np.array_equal(g["sorted_keys"], tr.sorted_keys), (mode, step)
            assert np.array_equal(g["sorted_ids"], tr.sorted_ids), (mode, step)
            pool.flush()
            pool.wait(0)
        pool.close()
