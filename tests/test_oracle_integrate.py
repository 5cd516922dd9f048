"""Pins of the oracle's leapfrog step (kick then drift, staggered velocities)
against what the mathematics fixes: rest without force, constant
acceleration from rest (closed form, exact in binary arithmetic), time
reversal, and the discrete invariant of the method on the harmonic
oscillator."""
import numpy as np

from oracle import oracle as O


def test_rest_without_force_is_unchanged():
    x = np.random.default_rng(1).normal(size=(50, 4)).astype(np.float32)
    v = np.zeros((50, 4), np.float32)
    x2, v2 = O.kick_drift(np.zeros((50, 4)), x, v, 0.25)
    assert np.array_equal(x2, x) and np.array_equal(v2, v)


def test_constant_acceleration_closed_form():
    # from rest, v_k = k a dt and x_k = x_0 + a dt^2 k (k + 1) / 2 exactly
    # (powers of two: no rounding)
    a, dt, steps = 0.5, 0.125, 12
    x = np.zeros((1, 4), np.float32)
    x[0, 3] = 1.0
    v = np.zeros((1, 4), np.float32)
    acc = np.array([[a, -2 * a, 0.0, 0.0]])
    for k in range(1, steps + 1):
        x, v = O.kick_drift(acc, x, v, dt)
        assert v[0, 0] == k * a * dt and v[0, 1] == -2 * k * a * dt
        assert x[0, 0] == a * dt * dt * k * (k + 1) / 2
        assert x[0, 1] == -2 * a * dt * dt * k * (k + 1) / 2
        assert x[0, 2] == 0.0 and x[0, 3] == 1.0     # mass kept


def test_kick_before_drift():
    # one step from rest with unit acceleration: the drift uses the kicked
    # velocity (x = a dt^2), not the old one (x = 0)
    x, v = O.kick_drift(np.array([[1.0, 0, 0, 0]]), np.zeros((1, 4), np.float32),
                        np.zeros((1, 4), np.float32), 0.5)
    assert x[0, 0] == 0.25 and v[0, 0] == 0.5


def test_time_reversal():
    # drift back with -dt, then kick with -dt at the same acceleration:
    # returns to the start (up to float32 rounding)
    g = np.random.default_rng(2)
    x = g.normal(size=(100, 4)).astype(np.float32)
    v = g.normal(size=(100, 4)).astype(np.float32)
    acc = g.normal(size=(100, 4))
    dt = 1e-2
    x1, v1 = O.kick_drift(acc, x, v, dt)
    x0 = (x1[:, :3].astype(np.float64) - v1[:, :3].astype(np.float64) * dt)
    v0 = v1[:, :3].astype(np.float64) - acc[:, :3] * dt
    np.testing.assert_allclose(x0, x[:, :3], rtol=0, atol=1e-6)
    np.testing.assert_allclose(v0, v[:, :3], rtol=0, atol=1e-6)


def test_harmonic_oscillator_invariant():
    # a = -x: the leapfrog step conserves 1/2 v(n-1/2) v(n+1/2) + 1/2 x(n)^2
    # exactly in exact arithmetic (a discrete invariant of the method); here
    # to float32 rounding over many periods
    x = np.array([[1.0, 0.0, 0.0, 1.0]], np.float32)
    v = np.array([[0.0, 0.0, 0.0, 0.0]], np.float32)
    dt = 0.05
    inv = []
    for _ in range(3000):
        xn, vm = float(x[0, 0]), float(v[0, 0])
        x, v = O.kick_drift(np.array([[-xn, 0.0, 0.0, 0.0]]), x, v, dt)
        inv.append(0.5 * vm * float(v[0, 0]) + 0.5 * xn * xn)
    inv = np.array(inv)
    assert np.abs(inv - 0.5).max() < 1e-5
