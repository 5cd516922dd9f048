"""Pins for the oracle's softened gravity sum (Section 4.1 force computation).

Each check rests on a fact other than the oracle's own formula: closed-form
two-body values, symmetry, Newton's third law, and the analytic Plummer
field (shell theorem)."""
import math

import numpy as np
import pytest

from paper_2008_05712_gb300 import inputs


def table(rows):
    return np.asarray(rows, dtype=np.float32)


def test_two_body_closed_form(orc):
    # source (m=2) at distance 3 on +x, eps^2 = 16 -> r^2 + eps^2 = 25 exactly:
    # a = m r / 125, phi = -m / 5
    t = table([[0, 0, 0, 0.5], [3, 0, 0, 2]])
    out = orc.gravity(t, [0], [1], 16.0)
    assert out[0, 0] == pytest.approx(2 * 3 / 125, abs=0, rel=1e-15)
    assert out[0, 1] == 0 and out[0, 2] == 0
    assert out[0, 3] == pytest.approx(-2 / 5, rel=1e-15)
    # reverse direction: the force on the source points back (-x) and scales
    # with the other mass
    out = orc.gravity(t, [1], [0], 16.0)
    assert out[0, 0] == pytest.approx(-0.5 * 3 / 125, rel=1e-15)
    assert out[0, 3] == pytest.approx(-0.5 / 5, rel=1e-15)


def test_two_body_diagonal_unsoftened(orc):
    # separation (1, 2, 2): |r| = 3, eps = 0 -> a = m r / 27
    t = table([[1, 1, 1, 1], [2, 3, 3, 4]])
    out = orc.gravity(t, [0], [1], 0.0)
    np.testing.assert_allclose(out[0, :3], 4 * np.array([1, 2, 2]) / 27, rtol=1e-15)
    assert out[0, 3] == pytest.approx(-4 / 3, rel=1e-15)


def test_self_term_is_zero_force(orc):
    t = table([[0.25, -1, 2, 3]])
    out = orc.gravity(t, [0], [0], 0.01)
    assert np.all(out[0, :3] == 0)
    assert out[0, 3] == pytest.approx(-3 / math.sqrt(0.01), rel=1e-15)


def test_octahedron_symmetry(orc):
    # six equal masses at +-d on each axis: zero field at the centre,
    # phi = -6 m / sqrt(d^2 + eps^2); at a vertex the field points to the centre
    d, m, eps2 = 2.0, 0.75, 0.25
    pts = [[0, 0, 0, 1]]
    for a in range(3):
        for s in (-1, 1):
            p = [0.0, 0.0, 0.0, m]
            p[a] = s * d
            pts.append(p)
    t = table(pts)
    out = orc.gravity(t, [0], list(range(1, 7)), eps2)
    assert np.max(np.abs(out[0, :3])) < 1e-15
    assert out[0, 3] == pytest.approx(-6 * m / math.sqrt(d * d + eps2), rel=1e-14)
    # vertex (+d,0,0): opposite vertex at distance 2d, four at distance d*sqrt2,
    # plus the centre mass 1 at distance d
    out = orc.gravity(t, [2], [0, 1, 3, 4, 5, 6], eps2)
    s2 = 2 * d * d + eps2
    ax = -(1.0 * d / (d * d + eps2) ** 1.5 + m * 2 * d / (4 * d * d + eps2) ** 1.5
           + 4 * m * d / s2 ** 1.5)
    assert out[0, 0] == pytest.approx(ax, rel=1e-14)
    assert abs(out[0, 1]) < 1e-15 and abs(out[0, 2]) < 1e-15


def test_newton_third_law(orc):
    x = inputs.plummer(512, 7)
    ids = np.arange(512, dtype=np.uint32)
    acc = orc.gravity(x, ids, ids, np.float32(1e-4))
    mom = (acc[:, :3] * x[:, 3:4].astype(np.float64)).sum(axis=0)
    scale = (np.abs(acc[:, :3]) * x[:, 3:4]).sum()
    assert np.max(np.abs(mom)) < 1e-13 * scale


def test_list_order_invariance(orc):
    x = inputs.plummer(300, 11)
    ids = np.arange(300, dtype=np.uint32)
    perm = np.random.default_rng(3).permutation(ids).astype(np.uint32)
    a = orc.gravity(x, ids[:20], ids, 1e-4)
    b = orc.gravity(x, ids[:20], perm, 1e-4)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


@pytest.mark.slow
def test_plummer_radial_profile(orc):
    # Shell theorem: the field at radius r of a spherical distribution is
    # -M(<r)/r^2.  For a Plummer sphere truncated at X = 0.999 of its mass
    # and renormalised to M = 1, M(<r) = r^3 (1 + r^2)^(-3/2) / 0.999.
    n = 12000
    x = inputs.plummer(n, 20080571)
    ids = np.arange(n, dtype=np.uint32)
    tgt = ids[::6]
    acc = orc.gravity(x, tgt, ids, 1e-8)   # tiny softening: self term finite
    p = x[tgt, :3].astype(np.float64)
    r = np.linalg.norm(p, axis=1)
    ar = (acc[:, :3] * p).sum(axis=1) / r
    for lo, hi in [(0.3, 0.6), (0.6, 1.0), (1.0, 1.6), (1.6, 3.0)]:
        sel = (r >= lo) & (r < hi)
        rr = r[sel]
        model = -(rr ** 3 * (1 + rr ** 2) ** -1.5 / 0.999) / rr ** 2
        ratio = ar[sel] / model
        # shot noise of a 12000-body realisation: a few percent per shell
        assert abs(ratio.mean() - 1) < 0.05, (lo, hi, ratio.mean())
