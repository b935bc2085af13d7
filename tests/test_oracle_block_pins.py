"""Pins of the oracle's block-time-step Hermite integrator (CPU only).

Individual power-of-two time steps are the usual partner of a jerk-based
integrator; the paper computes the jerk (Sec. 3) but does not describe its
stepping, so the scheme is written from Makino & Aarseth (1992).  Pinned by:
reduction to the (pinned) shared-step Hermite bit for bit when every step is
forced to dt_max; the block-time invariants (powers of two, commensurate
times, synchronisation at t_end); and convergence of a hierarchical triple,
whose members take different steps, towards an accurate shared-step reference.
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
