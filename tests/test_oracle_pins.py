"""Pins of the FP64 oracle to what the paper and the physics fix (CPU only).

The oracle is the reference for every GPU parity test, so it is checked here
against values it cannot produce by re-running its own formula: closed-form
static configurations, Newton's third law, exact power-of-two scaling, the
potential-gradient relation a = -grad(phi), Kepler two-body orbits against
Kepler's equation, exact momentum / angular-momentum conservation of KDK with
central pair forces, and the Plummer virial ratio.  A dropped term, a wrong
sign or exponent, a transposed operand or a missing j != i exclusion fails at
least one of these.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2509_19294_gb300 import ic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _eval(expr):
    return eval(expr, {"sqrt": math.sqrt, "__builtins__": {}})


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _golden()["cases"], ids=lambda c: c["name"])
@pytest.mark.parametrize("scale", [1.0, 0.5, 3.0])
def test_regular_configurations(oracle, case, scale):
    v = np.array(case["vertices"], np.float64).T * scale
    n = v.shape[1]
    edge = _eval(case.get("edge", "1")) * scale
    m = 0.7
    G = 1.3
    acc, pot = oracle.forces(v, np.full(n, m), eps=0.0, G=G)
    centroid = v.mean(axis=1)
    want_mag = _eval(case["a_mag"]) * G * m / edge ** 2
    want_phi = _eval(case["phi"]) * G * m / edge
    for i in range(n):
        d = centroid - v[:, i]
        want = want_mag * d / np.linalg.norm(d)
        np.testing.assert_allclose(acc[:, i], want, rtol=1e-14, atol=1e-14 * want_mag)
        assert pot[i] == pytest.approx(want_phi, rel=1e-14)


@pytest.mark.parametrize("tb", _golden()["two_body"], ids=lambda t: f"d{t['d']}_eps{t['eps']}")
def test_two_body_closed_form(oracle, tb):
    pos = np.array([[0.0, tb["d"]], [0.0, 0.0], [0.0, 0.0]])
    # rotate the pair off-axis so that all three components are exercised
    ang = 0.3
    rot = np.array([[math.cos(ang), -math.sin(ang), 0], [math.sin(ang), math.cos(ang), 0], [0, 0, 1]])
    rot = rot @ np.array([[1, 0, 0], [0, math.cos(0.7), -math.sin(0.7)], [0, math.sin(0.7), math.cos(0.7)]])
    pos = rot @ pos + np.array([[0.25], [-1.5], [2.0]])
    u = (pos[:, 1] - pos[:, 0]) / tb["d"]
    acc, pot = oracle.forces(pos, np.array(tb["m"]), eps=tb["eps"], G=tb["G"])
    np.testing.assert_allclose(acc[:, 0], tb["a0"] * u, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(acc[:, 1], tb["a1"] * u, rtol=1e-13, atol=1e-15)
    assert pot[0] == pytest.approx(tb["phi0"], rel=1e-14)
    assert pot[1] == pytest.approx(tb["phi1"], rel=1e-14)


def test_single_particle_feels_nothing(oracle):
    acc, pot = oracle.forces(np.array([[1.0], [2.0], [3.0]]), np.array([5.0]), eps=0.1)
    assert np.all(acc == 0.0) and pot[0] == 0.0


def test_self_term_excluded_with_softening(oracle):
    # with eps > 0 a self term would add -G m_i / eps to phi_i; two far-apart
    # particles make the difference obvious
    pos = np.array([[0.0, 1e6], [0.0, 0.0], [0.0, 0.0]])
    acc, pot = oracle.forces(pos, np.array([1.0, 1.0]), eps=0.5)
    assert abs(pot[0]) < 2e-6


def _random_system(n, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    pos = rng.normal(size=(3, n)) * spread
    mass = rng.uniform(0.1, 2.0, n)
    return pos, mass


@pytest.mark.parametrize("eps", [0.0, 0.05])
def test_newton_third_law(oracle, eps):
    pos, mass = _random_system(300, 11)
    acc, _ = oracle.forces(pos, mass, eps=eps)
    total = (acc * mass).sum(axis=1)
    scale = (np.abs(acc) * mass).sum()
    assert np.all(np.abs(total) <= 1e-14 * scale)


def test_power_of_two_scaling_is_exact(oracle):
    # positions x2, eps x2, masses x8  =>  a x2 and phi x4, bit for bit: every
    # operation scales by a power of two.  A wrong distance exponent breaks it.
    pos, mass = _random_system(64, 12)
    a1, p1 = oracle.forces(pos, mass, eps=0.03)
    a2, p2 = oracle.forces(pos * 2.0, mass * 8.0, eps=0.06)
    assert np.array_equal(a2, 2.0 * a1)
    assert np.array_equal(p2, 4.0 * p1)


def test_translation_and_permutation(oracle):
    pos, mass = _random_system(200, 13)
    a1, p1 = oracle.forces(pos, mass, eps=0.01)
    shift = np.array([[1e3], [-1e3], [1e3]])
    a2, p2 = oracle.forces(pos + shift, mass, eps=0.01)
    scale = np.abs(a1).max()
    assert np.abs(a2 - a1).max() <= 1e-9 * scale
    np.testing.assert_allclose(p2, p1, rtol=1e-10)
    perm = np.random.default_rng(5).permutation(200)
    a3, p3 = oracle.forces(pos[:, perm], mass[perm], eps=0.01)
    np.testing.assert_allclose(a3, a1[:, perm], rtol=1e-13, atol=1e-15 * scale)
    np.testing.assert_allclose(p3, p1[perm], rtol=1e-14)


def test_rows_match_full(oracle):
    pos, mass = _random_system(257, 14)
    a, p = oracle.forces(pos, mass, eps=0.02)
    rows = np.array([0, 5, 100, 256])
    ar, pr = oracle.forces_rows(pos, mass, eps=0.02, rows=rows)
    assert np.array_equal(ar, a[:, rows]) and np.array_equal(pr, p[rows])


@pytest.mark.parametrize("eps", [0.0, 0.2])
def test_acceleration_is_minus_potential_gradient(oracle, eps):
    # a massless probe feels a(r) = -grad phi(r) of the softened field
    pos, mass = _random_system(40, 15)
    probe = np.array([0.3, -0.2, 0.45])
    h = 1e-5
    P = np.concatenate([pos, probe[:, None]], axis=1)
    M = np.concatenate([mass, [0.0]])
    a0, _ = oracle.forces(P, M, eps=eps)
    grad = np.empty(3)
    for k in range(3):
        Pp = P.copy()
        Pm = P.copy()
        Pp[k, -1] += h
        Pm[k, -1] -= h
        _, pp = oracle.forces(Pp, M, eps=eps)
        _, pm = oracle.forces(Pm, M, eps=eps)
        grad[k] = (pp[-1] - pm[-1]) / (2 * h)
    np.testing.assert_allclose(a0[:, -1], -grad, rtol=1e-6, atol=1e-8)


def _kepler_relative(t, a, e, mu):
    """Relative position at time t from pericentre (Kepler's equation, Newton)."""
    n = math.sqrt(mu / a ** 3)
    M = n * t
    E = M if e < 0.8 else math.pi
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _kepler_run(oracle, e, steps_per_period, periods=1.0):
    m1, m2 = 0.3, 0.7
    mu = m1 + m2
    a = 1.0
    rp = a * (1 - e)
    vp = math.sqrt(mu * (1 + e) / rp)
    r = np.array([rp, 0.0, 0.0])
    v = np.array([0.0, vp, 0.0])
    pos = np.stack([-m2 / mu * r, m1 / mu * r], axis=1)
    vel = np.stack([-m2 / mu * v, m1 / mu * v], axis=1)
    T = 2 * math.pi * math.sqrt(a ** 3 / mu)
    nsteps = int(round(steps_per_period * periods))
    dt = periods * T / nsteps
    p, vv, _, _, dg = oracle.kdk(pos, vel, np.array([m1, m2]), eps=0.0, dt=dt, nsteps=nsteps,
                                 diag=True)
    rel = p[:, 1] - p[:, 0]
    want = _kepler_relative(periods * T, a, e, mu)
    return np.linalg.norm(rel - want), dg


@pytest.mark.parametrize("e", [0.0, 0.5])
def test_kepler_orbit_second_order(oracle, e):
    err1, _ = _kepler_run(oracle, e, 2000, periods=1.37)
    err2, dg = _kepler_run(oracle, e, 4000, periods=1.37)
    assert err2 < (2e-4 if e == 0 else 2e-3)
    ratio = err1 / err2
    assert 3.5 < ratio < 4.5, ratio          # leapfrog is second order
    # energy of the two-body problem: E = -G m1 m2 / (2a) at every output, to O(dt^2)
    m1, m2 = 0.3, 0.7
    assert np.abs(dg[:, 2] - (-m1 * m2 / 2.0)).max() < 1e-4


def test_kdk_conserves_momentum_and_angular_momentum(oracle):
    pos, mass = _random_system(24, 16)
    vel = np.random.default_rng(17).normal(size=(3, 24)) * 0.3
    _, _, _, _, dg = oracle.kdk(pos, vel, mass, eps=0.05, dt=1e-3, nsteps=200, diag=True)
    P0, L0 = dg[0, 3:6], dg[0, 6:9]
    scaleP = (mass * np.abs(vel).sum(axis=0)).sum()
    scaleL = (mass * np.linalg.norm(pos, axis=0) * np.linalg.norm(vel, axis=0)).sum()
    assert np.abs(dg[:, 3:6] - P0).max() <= 1e-13 * scaleP
    assert np.abs(dg[:, 6:9] - L0).max() <= 1e-12 * scaleL


def test_kdk_time_reversible(oracle):
    pos, mass = _random_system(16, 18)
    vel = np.random.default_rng(19).normal(size=(3, 16)) * 0.2
    p1, v1, _, _, _ = oracle.kdk(pos, vel, mass, eps=0.1, dt=2e-3, nsteps=50)
    p2, v2, _, _, _ = oracle.kdk(p1, -v1, mass, eps=0.1, dt=2e-3, nsteps=50)
    np.testing.assert_allclose(p2, pos, atol=1e-11)
    np.testing.assert_allclose(-v2, vel, atol=1e-11)


def test_energy_of_static_pair(oracle):
    # W = 1/2 sum m phi = -G m1 m2 / d ;  K = 1/2 sum m v^2
    pos = np.array([[0.0, 2.0], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [1.0, -2.0], [0.0, 0.0]])
    mass = np.array([1.0, 3.0])
    _, pot = oracle.forces(pos, mass, eps=0.0)
    e = oracle.energy(pos, vel, mass, pot)
    assert e[0] == pytest.approx(0.5 * (1 * 1 + 3 * 4))
    assert e[1] == pytest.approx(-1.5)
    np.testing.assert_allclose(e[3:6], [0.0, 1.0 - 6.0, 0.0])
    np.testing.assert_allclose(e[6:9], [0.0, 0.0, 3.0 * (2.0 * -2.0)])


def test_plummer_virial_and_henon_energy(oracle):
    n = 4096
    pos, vel, mass = ic.plummer(n, seed=1)
    _, pot = oracle.forces(pos, mass, eps=1e-3)
    e = oracle.energy(pos, vel, mass, pot)
    K, W, E = e[0], e[1], e[2]
    assert abs(2 * K / abs(W) - 1.0) < 5 / math.sqrt(n)
    assert abs(E - (-0.25)) < 0.02
    np.testing.assert_allclose(e[3:6], 0.0, atol=1e-12)


def test_plummer_mean_field(oracle):
    # large-N sanity: the radial acceleration follows a(r) = -G M r / (r^2 + b^2)^(3/2)
    n = 8192
    pos, _, mass = ic.plummer(n, seed=2)
    acc, _ = oracle.forces(pos, mass, eps=1e-3)
    r = np.linalg.norm(pos, axis=0)
    ar = (acc * pos).sum(axis=0) / r
    b = ic.HENON_R
    want = -r / (r * r + b * b) ** 1.5
    sel = (r > 0.3) & (r < 2.0)
    rel = np.median(np.abs(ar[sel] - want[sel]) / np.abs(want[sel]))
    assert rel < 0.05
