"""Pins of the oracle's jerk and Hermite integrator (CPU only).

The paper computes the acceleration together with its time derivative, the
jerk (Sec. 3).  The oracle's jerk is pinned by closed forms of two-body motion
along and across the separation, by the time derivative of the acceleration
along straight-line motion (central differences), by Newton's third law
(sum m_i jerk_i = 0), and by exact power-of-two scaling; the fourth-order
Hermite scheme by a Kepler orbit whose error falls 16-fold when dt halves.
"""
import math

import numpy as np
import pytest


def _rotated_pair(d, u_along, u_across, seed=3):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    pos = q @ np.array([[0.0, d], [0.0, 0.0], [0.0, 0.0]]) + np.array([[0.3], [-0.2], [1.1]])
    vel = q @ np.array([[0.0, u_along], [0.0, u_across], [0.0, 0.0]])
    return pos, vel, q


@pytest.mark.parametrize("eps", [0.0, 0.7])
def test_two_body_jerk_closed_forms(oracle, eps):
    m = np.array([1.0, 3.0])
    d, G = 2.0, 1.5
    # motion along the separation: jerk_0 = G m1 u (eps^2 - 2 d^2) / (d^2 + eps^2)^(5/2)
    pos, vel, q = _rotated_pair(d, 0.8, 0.0)
    _, j, _ = oracle.forces_jerk(pos, vel, m, eps, G)
    want = G * 3.0 * 0.8 * (eps ** 2 - 2 * d * d) / (d * d + eps ** 2) ** 2.5
    np.testing.assert_allclose(j[:, 0], want * q[:, 0], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(j[:, 1], -(1.0 / 3.0) * want * q[:, 0], rtol=1e-13, atol=1e-15)
    # motion across the separation: r . v = 0, jerk_0 = G m1 v / (d^2 + eps^2)^(3/2)
    pos, vel, q = _rotated_pair(d, 0.0, 0.6)
    _, j, _ = oracle.forces_jerk(pos, vel, m, eps, G)
    want = G * 3.0 * 0.6 / (d * d + eps ** 2) ** 1.5
    np.testing.assert_allclose(j[:, 0], want * q[:, 1], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("eps", [0.0, 0.05])
def test_jerk_is_the_time_derivative_of_the_acceleration(oracle, eps):
    rng = np.random.default_rng(21)
    n = 30
    pos = rng.normal(size=(3, n))
    vel = rng.normal(size=(3, n)) * 0.5
    mass = rng.uniform(0.2, 1.0, n)
    a0, j0, p0 = oracle.forces_jerk(pos, vel, mass, eps)
    h = 1e-5
    ap, _ = oracle.forces(pos + h * vel, mass, eps)
    am, _ = oracle.forces(pos - h * vel, mass, eps)
    fd = (ap - am) / (2 * h)
    scale = np.abs(j0).max()
    np.testing.assert_allclose(j0, fd, rtol=1e-6, atol=1e-7 * scale)
    a_ref, p_ref = oracle.forces(pos, mass, eps)
    np.testing.assert_allclose(a0, a_ref, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(p0, p_ref, rtol=1e-14)


def test_jerk_newton_third_law_and_scaling(oracle):
    rng = np.random.default_rng(22)
    n = 200
    pos = rng.normal(size=(3, n))
    vel = rng.normal(size=(3, n))
    mass = rng.uniform(0.1, 2.0, n)
    a, j, p = oracle.forces_jerk(pos, vel, mass, 0.03)
    total = (j * mass).sum(axis=1)
    assert np.all(np.abs(total) <= 1e-13 * (np.abs(j) * mass).sum())
    # x, v, eps x2 and m x8: a x2, jerk x2, phi x4, bit for bit
    a2, j2, p2 = oracle.forces_jerk(pos * 2, vel * 2, mass * 8, 0.06)
    assert np.array_equal(a2, 2 * a) and np.array_equal(j2, 2 * j) and np.array_equal(p2, 4 * p)


def _kepler_hermite(oracle, steps_per_period, e=0.5, periods=1.37):
    m1, m2 = 0.3, 0.7
    mu = m1 + m2
    rp = 1 - e
    vp = math.sqrt(mu * (1 + e) / rp)
    r = np.array([rp, 0.0, 0.0])
    v = np.array([0.0, vp, 0.0])
    pos = np.stack([-m2 / mu * r, m1 / mu * r], axis=1)
    vel = np.stack([-m2 / mu * v, m1 / mu * v], axis=1)
    T = 2 * math.pi / math.sqrt(mu)
    nsteps = int(round(steps_per_period * periods))
    dt = periods * T / nsteps
    p, _, _, _, _, dg = oracle.hermite(pos, vel, np.array([m1, m2]), 0.0, dt, nsteps, diag=True)
    # Kepler's equation for the final relative position
    M = math.sqrt(mu) * periods * T
    E = M
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    want = np.array([math.cos(E) - e, math.sqrt(1 - e * e) * math.sin(E), 0.0])
    return np.linalg.norm((p[:, 1] - p[:, 0]) - want), dg


def test_hermite_is_fourth_order(oracle):
    err1, _ = _kepler_hermite(oracle, 1000)
    err2, dg = _kepler_hermite(oracle, 2000)
    ratio = err1 / err2
    assert 13.0 < ratio < 19.0, ratio
    assert err2 < 1e-6
    assert np.abs(dg[:, 2] - (-0.3 * 0.7 / 2.0)).max() < 1e-7


def test_rows_variant_indexes_the_same_evaluation(oracle):
    # the sampled-row form (used at full size) returns exactly the full
    # evaluation's values at those rows, in the order asked
    rng = np.random.default_rng(77)
    n = 40
    pos, vel = rng.normal(size=(3, n)), rng.normal(size=(3, n))
    mass = rng.uniform(0.5, 1.5, n) / n
    a, j, p = oracle.forces_jerk(pos, vel, mass, 0.05)
    rows = np.array([7, 0, 39, 7, 21])
    ar, jr, pr = oracle.forces_jerk_rows(pos, vel, mass, 0.05, rows)
    assert np.array_equal(ar, a[:, rows]) and np.array_equal(jr, j[:, rows])
    assert np.array_equal(pr, p[rows])
