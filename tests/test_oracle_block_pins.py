"""Pins of the oracle's block-time-step Hermite integrator (CPU only).

Individual power-of-two time steps are the usual partner of a jerk-based
integrator; the paper computes the jerk (Sec. 3) but does not describe its
stepping, so the scheme is written from Makino & Aarseth (1992).  Pinned by:
reduction to the (pinned) shared-step Hermite bit for bit when every step is
forced to dt_max; the block-time invariants (powers of two, commensurate
times, synchronisation at t_end); convergence of a hierarchical triple, whose
members take different steps, towards an accurate shared-step reference; and
the step rules themselves:
* Aarseth's criterion from the Hermite interpolation is exact when the
  acceleration history is a cubic in time (the interpolant then reproduces
  the second derivative at the step end and the third derivative exactly);
* on a circular binary every derivative has a closed-form magnitude,
  |a^(k)| = omega^(k+2) r, so the first step rule eta_s |a| / |a'| is
  eta_s / omega and the criterion is sqrt(eta) / omega: the oracle's steps
  must be the powers of two just below those values.
"""
import numpy as np
import pytest


def _triple():
    # a tight binary (separation 0.02) and a distant third body
    pos = np.array([[-0.01, 0.01, 1.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.1]])
    vb = np.sqrt(1.0 / 0.02) / 2          # circular binary, total mass 1 in the pair... roughly
    vel = np.array([[0.0, 0.0, 0.0], [-vb, vb, 0.6], [0.0, 0.0, 0.0]])
    mass = np.array([0.5, 0.5, 0.01])
    return pos, vel, mass


def test_equal_steps_reduce_to_shared_hermite(oracle):
    rng = np.random.default_rng(31)
    n = 24
    pos = rng.normal(size=(3, n))
    vel = rng.normal(size=(3, n)) * 0.3
    mass = rng.uniform(0.2, 1.0, n) / n
    dtm = 2.0 ** -8
    # eta huge: every particle keeps dt_max; eta_s huge: it starts there
    bp, bv, ba, bj, _, dt, blocks, evals = oracle.block_hermite(pos, vel, mass, 0.05, 16 * dtm, dtm,
                                                              2.0 ** -30, 1e30, 1e30)
    sp, sv, sa, sj, _, _ = oracle.hermite(pos, vel, mass, 0.05, dtm, 16)
    assert blocks == 16 and evals == 16 * n and np.all(dt == dtm)
    assert np.array_equal(bp, sp) and np.array_equal(bv, sv)
    assert np.array_equal(ba, sa) and np.array_equal(bj, sj)


def test_block_invariants_and_synchronisation(oracle):
    pos, vel, mass = _triple()
    t_end, dtm = 2.0 ** -3, 2.0 ** -5
    bp, bv, ba, bj, _, dt, blocks, evals = oracle.block_hermite(pos, vel, mass, 0.0, t_end, dtm,
                                                              2.0 ** -24, 0.02, 0.01)
    lg = np.log2(dt)
    assert np.all(lg == np.round(lg)) and np.all(dt <= dtm)
    # the binary members take far smaller steps than the distant body
    assert dt[2] > 8 * max(dt[0], dt[1])
    # evaluations: the distant body is evaluated far less often than the binary
    assert evals < blocks * 3
    # at t_end everybody is synchronised: the stored a, jerk (taken at each
    # particle's last predicted state) agree with a fresh evaluation to the
    # O(dt^4) size of the last correction; a particle left at an earlier time
    # would be off by |jerk| * dt, orders of magnitude more
    fa, fj, _ = oracle.forces_jerk(bp, bv, mass, 0.0)
    rel = lambda x, y: np.linalg.norm(x - y, axis=0) / np.linalg.norm(y, axis=0)
    assert rel(ba, fa).max() < 1e-4 and rel(bj, fj).max() < 1e-3, (rel(ba, fa), rel(bj, fj))


def test_block_steps_converge_to_accurate_reference(oracle):
    pos, vel, mass = _triple()
    t_end = 2.0 ** -3
    ref, *_ = oracle.hermite(pos, vel, mass, 0.0, 2.0 ** -16, int(t_end * 2 ** 16))
    errs, steps = [], []
    for eta in (0.08, 0.005):
        bp, *_, dt, _, _ = oracle.block_hermite(pos, vel, mass, 0.0, t_end, 2.0 ** -5, 2.0 ** -24,
                                                eta, eta / 2)
        errs.append(np.abs(bp - ref).max())
        steps.append(dt[0])
    # eta / 16 quarters the binary's step (dt ~ eta^(1/2)); a fourth-order
    # scheme then cuts the error by ~4^4
    assert steps[1] == steps[0] / 4, steps
    assert errs[1] < errs[0] / 100, errs
    assert errs[1] < 1e-6


def test_criterion_is_exact_for_a_cubic_acceleration_history(oracle):
    # a(t) = c0 + c1 t + c2 t^2 + c3 t^3: a'(h), a''(h) = 2 c2 + 6 c3 h and
    # a'''(h) = 6 c3 are exact, and the criterion takes a'' at the step END
    rng = np.random.default_rng(41)
    nrm = np.linalg.norm
    eta = 0.02
    for h in (0.5, 2.0 ** -3, 2.0 ** -6):
        for _ in range(4):
            c0, c1, c2, c3 = rng.normal(size=(4, 3))
            a0, j0 = c0, c1
            a1 = c0 + c1 * h + c2 * h ** 2 + c3 * h ** 3
            j1 = c1 + 2 * c2 * h + 3 * c3 * h ** 2
            s2, s3 = 2 * c2 + 6 * c3 * h, 6 * c3
            want = np.sqrt(eta * (nrm(a1) * nrm(s2) + nrm(j1) ** 2) / (nrm(j1) * nrm(s3) + nrm(s2) ** 2))
            got = oracle.aarseth_step(a0, j0, a1, j1, h, eta)
            assert got == pytest.approx(want, rel=1e-9), (h, got, want)


def _circular_binary(omega):
    # equal masses 1/2 (G = 1, total mass 1) at separation d with
    # omega^2 = 1 / d^3: each body moves on a circle of radius d/2
    d = omega ** (-2.0 / 3.0)
    v = omega * d / 2
    pos = np.array([[d / 2, -d / 2], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [v, -v], [0.0, 0.0]])
    return pos, vel, np.array([0.5, 0.5])


def test_first_steps_on_a_circular_binary(oracle):
    # |a| / |a'| = 1 / omega for each body: the first step is the largest
    # power of two <= eta_s / omega (here 2^-9.5, so 2^-10); t_end = 0 stops
    # before the first block step
    omega = 8.0
    pos, vel, mass = _circular_binary(omega)
    eta_s = omega * 2.0 ** -9.5
    *_, dt, blocks, _ = oracle.block_hermite(pos, vel, mass, 0.0, 0.0, 2.0 ** -3, 2.0 ** -30, 0.02,
                                             eta_s)
    assert blocks == 0 and np.all(dt == 2.0 ** -10), dt


def test_circular_binary_settles_on_the_closed_form_step(oracle):
    # sqrt(eta) / omega = 2^-7.5: from first steps of 2^-10 the doubling rule
    # climbs one level per allowed step to 2^-8 and stays there (2^-7 is above
    # the criterion); two orbits (t_end = 1.5, omega t = 12)
    omega = 8.0
    pos, vel, mass = _circular_binary(omega)
    eta = (omega * 2.0 ** -7.5) ** 2
    eta_s = omega * 2.0 ** -9.5
    bp, bv, *_, dt, blocks, evals = oracle.block_hermite(pos, vel, mass, 0.0, 1.5, 2.0 ** -3,
                                                         2.0 ** -30, eta, eta_s)
    assert np.all(dt == 2.0 ** -8), dt
    # every step after the climb is 2^-8: a few climbing steps plus 1.5 / 2^-8
    assert 1.5 * 2 ** 8 <= blocks <= 1.5 * 2 ** 8 + 4, blocks
    # and the orbit stays circular to the fourth-order scheme's accuracy
    r = np.linalg.norm(bp[:, 0] - bp[:, 1])
    assert abs(r - omega ** (-2.0 / 3.0)) < 1e-7, r
