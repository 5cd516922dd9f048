"""Pins of the oracle's Ewald correction (periodic gravity minus the plain
point-mass term) against what the mathematics fixes: independence of the
splitting parameter alpha, zero periodic force at the symmetry points of
the cube, the simple-cubic Madelung constant at zero separation, the force
as minus the gradient of the potential, linearity in the mass and the
periodicity of the full interaction."""
import numpy as np
import pytest

from oracle import oracle as O

# simple-cubic lattice sum with a neutralising background:
# psi(r) - 1/r -> XI / L as r -> 0 (the Ewald self term of a cubic lattice)
XI = -2.837297479480620


def table(points, m=1.0):
    t = np.zeros((len(points) + 1, 4), np.float32)
    t[0] = (0.0, 0.0, 0.0, m)
    for i, p in enumerate(points):
        t[i + 1, :3] = p
        t[i + 1, 3] = 1.0
    return t


def corr(points, L=1.0, m=1.0, **kw):
    t = table(points, m)
    return O.ewald(t, np.arange(1, len(points) + 1), [0], L, **kw)


def test_alpha_independence():
    g = np.random.default_rng(3)
    pts = g.uniform(-0.5, 0.5, size=(40, 3)).astype(np.float32)
    for L in (1.0, 2.5):
        a = corr(pts * L, L)
        b = corr(pts * L, L, alpha=3.0 / L, nrep=3, hcut2=30)
        c = corr(pts * L, L, alpha=1.6 / L, nrep=3, hcut2=10)
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-9 / L ** 2)
        np.testing.assert_allclose(a, c, rtol=1e-8, atol=1e-8 / L ** 2)


@pytest.mark.parametrize("p", [(0.5, 0, 0), (0, 0.5, 0), (0.5, 0.5, 0), (0.5, 0.5, 0.5)])
def test_symmetry_points_feel_no_periodic_force(p):
    # the periodic force vanishes; the correction cancels the plain term
    r = np.array(p, np.float64)
    a = corr([p])[0]
    np.testing.assert_allclose(a[:3], r / np.linalg.norm(r) ** 3, rtol=1e-9, atol=1e-9)


def test_madelung_constant_at_zero_separation():
    for L in (1.0, 3.0):
        a = corr([(0.0, 0.0, 0.0)], L, m=2.0)[0]
        assert a[3] == pytest.approx(-2.0 * XI / L, rel=1e-12)
        assert np.abs(a[:3]).max() < 1e-12


def test_force_is_minus_gradient_of_potential():
    g = np.random.default_rng(4)
    h = 2.0 ** -12
    for p in g.uniform(-0.45, 0.45, size=(10, 3)):
        p = np.round(p * 2 ** 20) / 2 ** 20          # exact in float32
        a = corr([p])[0]
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            up = corr([p + e])[0][3]
            dn = corr([p - e])[0][3]
            # a = -grad(phi) of the correction (phi_corr = -psi + 1/r, a_corr = grad psi + r/r^3)
            assert a[c] == pytest.approx(-(up - dn) / (2 * h), rel=1e-5, abs=1e-6)


def test_linear_in_mass_and_periodic():
    p = tuple(np.round(np.array([0.21, -0.13, 0.34]) * 2 ** 20) / 2 ** 20)   # exact in float32
    a1 = corr([p], m=1.0)[0]
    a3 = corr([p], m=3.0)[0]
    np.testing.assert_allclose(a3, 3 * a1, rtol=1e-14)
    # full periodic interaction = correction + plain term; periodic in r
    def full(q):
        q = np.array(q, np.float64)
        c = corr([tuple(q)])[0]
        r = np.linalg.norm(q)
        return c[:3] - q / r ** 3, c[3] - 1.0 / r
    f0, u0 = full(p)
    f1, u1 = full((p[0] - 1.0, p[1], p[2]))
    # equal up to the truncation of the sums (images |n| <= 2, |h|^2 <= 10)
    np.testing.assert_allclose(f1, f0, rtol=1e-8, atol=1e-8)
    assert u1 == pytest.approx(u0, rel=1e-8)
