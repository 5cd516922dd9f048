"""GPU tests of the leapfrog step around the force computation (Section 4.1):
bit-exact against the oracle on given accelerations, the new positions
reach the pool, and one device-resident N-body step (tree, lists, batched
interaction, per-id totals as accelerations, kick-drift) against the FP64
oracle's step."""
import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs
from gpu_util import EPS2, TOL, make_pool, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    return gcharm


def test_kick_drift_bit_exact(gc, orc):
    g = np.random.default_rng(71)
    n = 5000
    x = g.normal(size=(n, 4)).astype(np.float32)
    v = g.normal(size=(n, 4)).astype(np.float32)
    acc = g.normal(size=(n, 4)) * 10.0
    dt = 0.0123
    pool = make_pool(gc, torch, n, n)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    xd = torch.from_numpy(x.copy()).cuda()
    vd = torch.from_numpy(v.copy()).cuda()
    ad = torch.from_numpy(acc).cuda()
    pool.kick_drift(ad, xd, vd, dt)
    torch.cuda.synchronize()
    x_ref, v_ref = orc.kick_drift(acc, x, v, dt)
    assert np.array_equal(xd.cpu().numpy(), x_ref)
    assert np.array_equal(vd.cpu().numpy(), v_ref)
    # the pool holds the new positions: a two-body task sees them
    to = np.array([0, 1], np.uint64)
    so = np.array([0, 1], np.uint64)
    b = pool.submit_csr(np.zeros(1, np.uint32), to, np.array([0], np.uint32), so,
                        np.array([1], np.uint32))
    pool.flush()
    pool.wait(b)
    ref = orc.gravity_batch(x_ref, to, np.array([0], np.uint32), so, np.array([1], np.uint32),
                            EPS2)
    assert rel_l2(pool.values()[:, :3], ref[:, :3]) <= TOL
    pool.close()


def test_device_resident_nbody_step(gc, orc):
    n = 8192
    x = inputs.plummer(n, 72)
    dt = 1e-3
    pool = make_pool(gc, torch, 3 * n + 64, 3 * n + 64)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    xd = torch.from_numpy(x.copy()).cuda()
    vd = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    pool.reset_totals()
    pool.build_nbody(xd, 32, 7, 10)
    pool.flush()
    pool.kick_drift(pool.totals_device_ptr(), xd, vd, dt)
    torch.cuda.synchronize()
    # the oracle's step: tree, lists, FP64 gravity, kick-drift
    tr = orc.Tree(x)
    tab = np.concatenate([x, tr.node_table()])
    to, tg = tr.bucket_targets()
    lo, li = tr.lists(7, 10)
    rows = orc.gravity_batch(tab, to, tg, lo, li, EPS2)
    acc = np.zeros((n, 4))
    acc[tg] = rows
    x_ref, v_ref = orc.kick_drift(acc, x, np.zeros((n, 4), np.float32), dt)
    v_gpu = vd.cpu().numpy()
    assert rel_l2(v_gpu[:, :3], v_ref[:, :3]) <= TOL
    per = np.linalg.norm(v_gpu[:, :3] - v_ref[:, :3], axis=1) / np.linalg.norm(v_ref[:, :3],
                                                                              axis=1)
    assert np.percentile(per, 99) <= TOL
    # positions: a few float32 ulps of each coordinate at most
    x_gpu = xd.cpu().numpy()
    ulp = np.spacing(np.abs(x_ref[:, :3]).astype(np.float32))
    assert np.all(np.abs(x_gpu[:, :3] - x_ref[:, :3]) <= 4 * ulp)
    assert np.array_equal(x_gpu[:, 3], x[:, 3])
    pool.close()
