"""Leapfrog, diagnostics, graph replay and conservation on the GPU (parity with the oracle)."""
import numpy as np
import pytest
import torch

import paper_2509_19294_gb300 as nb
from paper_2509_19294_gb300 import ic
from tests import metrics
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_19294_gb300 import build
    build.build()
    nb.load()
    torch.cuda.init()


def run_steps(pos, vel, mass, eps, dt, nsteps, mode, chunks=1, flags=0, offsets=None, **kw):
    """Advance on the GPU; returns (pos, vel, acc, pot, diag[nsteps, ncl, 9])."""
    n = mass.shape[0]
    ctx = nb.nbody_init(n, eps, mode=mode, cluster_offsets=offsets, flags=flags, **kw)
    p, v, m = dev(pos), dev(vel), dev(mass)
    acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    nb.nbody_forces(ctx, p, m, acc, pot)
    per = nsteps // chunks
    diags = []
    for _ in range(chunks):
        d = torch.empty((per, ctx.n_clusters, 9), dtype=torch.float64, device="cuda")
        nb.nbody_step(ctx, p, v, m, acc, pot, dt, per, d)
        diags.append(host(d))
    out = host(p), host(v), host(acc), host(pot), np.concatenate(diags)
    nb.nbody_destroy(ctx)
    return out


def assert_trajectory_close(gp, gv, rp, rv, ra, dt, nsteps, rel=1e-4):
    """An acceleration error of at most rel * max|a| per evaluation moves a
    velocity by at most nsteps * dt * rel * max|a| and a position by at most
    nsteps^2 * dt^2 * rel * max|a| (KDK applies each force once per step)."""
    amax = np.abs(ra).max()
    assert np.abs(gv - rv).max() <= nsteps * dt * rel * amax
    assert np.abs(gp - rp).max() <= nsteps ** 2 * dt ** 2 * rel * amax


def test_f64_kdk_plummer_1024_10_steps(oracle):
    pos, vel, mass = ic.plummer(1024, seed=1)
    gp, gv, ga, gpot, gd = run_steps(pos, vel, mass, 0.01, 1e-3, 10, nb.NBODY_F64)
    rp, rv, ra, rpot, rd = oracle.kdk(pos, vel, mass, 0.01, 1e-3, 10, diag=True)
    np.testing.assert_allclose(gp, rp, rtol=0, atol=1e-13)
    np.testing.assert_allclose(gv, rv, rtol=0, atol=1e-12)
    assert metrics.rel_acc_errors(ga, ra).max() <= 1e-11
    np.testing.assert_allclose(gd[:, 0, :], rd[1:, :], rtol=1e-11, atol=1e-13)


def test_f32c_kdk_tracks_oracle(oracle):
    pos, vel, mass = ic.plummer(4096, seed=3)
    gp, gv, ga, _, gd = run_steps(pos, vel, mass, 0.01, 1e-3, 20, nb.NBODY_F32C, reorder_every=5)
    rp, rv, ra, _, rd = oracle.kdk(pos, vel, mass, 0.01, 1e-3, 20, diag=True)
    assert_trajectory_close(gp, gv, rp, rv, ra, 1e-3, 20)
    s = metrics.summary(ga, ra)
    assert s["median"] <= 1e-6 and s["max"] <= 1e-4, s
    np.testing.assert_allclose(gd[:, 0, 2], rd[1:, 2], rtol=1e-6)  # W inherits phi's 1e-6


@pytest.mark.parametrize("mode", [nb.NBODY_F32C, nb.NBODY_F64])
def test_graph_replay_equals_eager(mode):
    pos, vel, mass = ic.plummer(3000, seed=4)
    g = run_steps(pos, vel, mass, 0.01, 1e-3, 12, mode, chunks=3, reorder_every=4)
    e = run_steps(pos, vel, mass, 0.01, 1e-3, 12, mode, chunks=3, reorder_every=4,
                  flags=nb.NBODY_FLAG_NO_GRAPH)
    for x, y in zip(g, e):
        assert np.array_equal(x, y)


def test_chunked_steps_equal_one_call():
    pos, vel, mass = ic.plummer(2000, seed=5)
    a = run_steps(pos, vel, mass, 0.01, 1e-3, 8, nb.NBODY_F32C, chunks=1)
    b = run_steps(pos, vel, mass, 0.01, 1e-3, 8, nb.NBODY_F32C, chunks=4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_host_buffers_through_step(oracle):
    pos, vel, mass = ic.plummer(1500, seed=6)
    n = 1500
    with nb.nbody_init(n, 0.01) as ctx:
        p, v = pos.copy(), vel.copy()
        acc, pot = np.empty((3, n)), np.empty(n)
        nb.nbody_forces(ctx, p, mass, acc, pot)
        diag = np.empty((5, 1, 9))
        nb.nbody_step(ctx, p, v, mass, acc, pot, 1e-3, 5, diag)
    d = run_steps(pos, vel, mass, 0.01, 1e-3, 5, nb.NBODY_F32C)
    for x, y in zip((p, v, acc, pot, diag), d):
        assert np.array_equal(x, y)


def test_conservation_f32c_within_twice_f64():
    # Plummer, eps = 1e-3, equal masses, 200 steps in four chunks: the FP32C
    # run's |dE/E| drift stays within 2x of the FP64 GPU run's over the same
    # steps, with no floor (the FP64 drift, ~6e-8, is far above the FP32C
    # energy jitter).  Momentum: FP32 pair terms break Newton's third law only
    # at the rounding level, so |dP| <= steps * dt * 1e-6 * sum m|a| (the
    # median relative force error target as the per-pair asymmetry bound);
    # the FP64 path's |dP| is pure roundoff and is no scale for it
    pos, vel, mass = ic.plummer(8192, seed=3)
    res = {}
    for mode in (nb.NBODY_F32C, nb.NBODY_F64):
        *_, acc, _, d = run_steps(pos, vel, mass, 1e-3, 1e-4, 200, mode, chunks=4, reorder_every=10)
        res[mode] = (d[:, 0, :], acc)
    (e32, a32), (e64, _) = res[nb.NBODY_F32C], res[nb.NBODY_F64]
    drift32 = np.abs(e32[:, 2] - e32[0, 2]).max() / abs(e32[0, 2])
    drift64 = np.abs(e64[:, 2] - e64[0, 2]).max() / abs(e64[0, 2])
    assert drift32 <= 2 * drift64, (drift32, drift64)
    dP32 = np.abs(e32[:, 3:6] - e32[0, 3:6]).max()
    assert dP32 <= 200 * 1e-4 * 1e-6 * (mass * np.linalg.norm(a32, axis=0)).sum(), dP32


def test_ensemble_steps_match_oracle(oracle):
    ens = ic.ensemble(6, seed=7, n_min=256, n_max=1500)
    gp, gv, ga, gpot, gd = run_steps(ens.pos, ens.vel, ens.mass, ens.eps, 1e-3, 5, nb.NBODY_F32C,
                                     offsets=ens.offsets, reorder_every=2)
    for c in range(6):
        b, e = ens.offsets[c], ens.offsets[c + 1]
        rp, rv, ra, _, rd = oracle.kdk(ens.pos[:, b:e], ens.vel[:, b:e], ens.mass[b:e], ens.eps[c],
                                       1e-3, 5, diag=True)
        assert_trajectory_close(gp[:, b:e], gv[:, b:e], rp, rv, ra, 1e-3, 5)
        s = metrics.summary(ga[:, b:e], ra)
        assert s["median"] <= 1e-6 and s["max"] <= 1e-4, (c, s)
        np.testing.assert_allclose(gd[:, c, 2], rd[1:, 2], rtol=1e-6)  # W inherits phi's 1e-6
