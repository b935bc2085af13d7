"""The five reference workloads through the CUDA path, checked against the oracle (GPU).

C1  Plummer N=1024, eps=0.01, KDK dt=1e-3, 10 steps, FP64 path: a, phi and E
    each step against the oracle's own leapfrog.
C2  N=16384 uniform sphere and Plummer, log-uniform masses, eps=0.005
    (covered in test_gpu_parity.py::test_f32c_16384_log_uniform_masses).
C3  Plummer N=131072, eps=1e-3, dt=1e-4, graph-replayed steps: the FP32C and
    FP64 GPU paths agree step by step on E and P over 10 steps, and over 100
    steps the FP32C |dE/E| drift is within twice the FP64 path's (the
    1000-step run is in bench.py's drift section and opt-in here with
    NBODY_LONG=1: about 13 minutes of FP64 work).
C4  512 clusters, N_c ~ U{256..8192}, eps_c = 0.01 N_c^(-1/3): every cluster's
    forces against the oracle, then steps with per-cluster diagnostics; over
    100 steps every cluster's FP32C |dE/E| drift is within twice its FP64
    path's.

The drift gates have no additive floor.  They sit where the FP64 path's own
drift exceeds the FP32C energy's evaluation-to-evaluation jitter (about 2e-10
of |E| at N = 131072: FP32 pairwise rounding of the potential, which no
summation order removes); over fewer steps the F32C energy is checked against
the FP64 path's step by step instead.
C5  two Plummer spheres of 524288 on a head-on approach, eps=1e-3: sampled rows
    of the full-size launch (the configuration bench.py times) against the
    oracle row by row.
Paper scale (N=102400, the paper's particle count): acceleration, jerk and
    potential of the launch configuration bench.py times, sampled rows against
    the oracle; the block-step workload's state after its first dt_max.

FP32C tolerance: per-particle relative acceleration error median <= 1e-6 and
max <= 1e-4, potential likewise, and the paper's 0.05 % bound (each component)
against the particle's own force magnitude and, at C5 and paper scale, against
the RMS force magnitude (see tests/metrics.py).  At C4 the RMS reading is
reported per cluster, not gated: a particle in a close encounter has |a_i| far
above its cluster's RMS.
"""
import os

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


def check_f32c(a, p, ra, rp, rms=True):
    s = metrics.summary(a, ra, p, rp)
    assert s["median"] <= 1e-6 and s["max"] <= 1e-4, s
    assert s["pot_median"] <= 1e-6 and s["pot_max"] <= 1e-4, s
    assert s["paper"] <= 5e-4, s
    if rms:
        assert s["paper_rms"] <= 5e-4, s
    return s


def test_c1_fp64_steps_match_oracle_each_step(oracle):
    pos, vel, mass = ic.plummer(1024, seed=1)
    n = 1024
    with nb.nbody_init(n, 0.01, mode=nb.NBODY_F64) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, p, m, acc, pot)
        rp, rv, ra, rpot = pos, vel, None, None
        for step in range(10):
            d = torch.empty((1, 1, 9), dtype=torch.float64, device="cuda")
            nb.nbody_step(ctx, p, v, m, acc, pot, 1e-3, 1, d)
            rp, rv, ra, rpot, rd = oracle.kdk(rp, rv, mass, 0.01, 1e-3, 1, acc=ra, pot=rpot,
                                             diag=True)
            assert metrics.rel_acc_errors(host(acc), ra).max() <= 1e-11, step
            assert metrics.rel_pot_errors(host(pot), rpot).max() <= 1e-11, step
            np.testing.assert_allclose(host(d)[0, 0], rd[1], rtol=1e-11, atol=1e-14)


def energy_track(pos, vel, mass, eps, dt, nsteps, mode, offsets=None, reorder_every=10):
    """[nsteps + 1, clusters, 9] diagnostics at t = 0 and after every step."""
    n = mass.shape[0]
    with nb.nbody_init(n, eps, mode=mode, cluster_offsets=offsets, reorder_every=reorder_every) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, p, m, acc, pot)
        e0 = nb.nbody_energy(ctx, p, v, m, pot)
        d = torch.empty((nsteps, ctx.n_clusters, 9), dtype=torch.float64, device="cuda")
        nb.nbody_step(ctx, p, v, m, acc, pot, dt, nsteps, d)
        return np.concatenate([e0[None], host(d)])


def drift(e):
    """Per cluster: max over steps of |E(t) - E(0)| / |E(0)|, E with the path's own phi."""
    return np.abs(e[:, :, 2] - e[0, :, 2]).max(axis=0) / np.abs(e[0, :, 2])


def test_c3_fp32c_tracks_fp64_each_step():
    # 10 steps: the FP64 path drifts ~5e-11, below the FP32C energy's
    # evaluation jitter, so E itself is compared step by step (the FP32C
    # potential's bias and jitter: measured 1.0-1.1e-8 of |E|)
    pos, vel, mass = ic.plummer(131072, seed=3)
    e32 = energy_track(pos, vel, mass, 1e-3, 1e-4, 10, nb.NBODY_F32C)[:, 0]
    e64 = energy_track(pos, vel, mass, 1e-3, 1e-4, 10, nb.NBODY_F64)[:, 0]
    assert np.abs(e32[:, 2] - e64[:, 2]).max() / abs(e64[0, 2]) <= 3e-8, (e32[:, 2], e64[:, 2])
    assert np.abs(e32[:, 3:6] - e64[:, 3:6]).max() <= 1e-9              # P
    assert np.abs(e32[:, 6:9] - e64[:, 6:9]).max() <= 1e-9              # L


def test_c3_100_steps_drift_within_twice_fp64():
    # the FP64 path's own drift over 100 steps (~1.4e-9) exceeds the FP32C
    # jitter: the twice-the-FP64-drift target applies with no floor
    pos, vel, mass = ic.plummer(131072, seed=3)
    d32 = drift(energy_track(pos, vel, mass, 1e-3, 1e-4, 100, nb.NBODY_F32C))[0]
    d64 = drift(energy_track(pos, vel, mass, 1e-3, 1e-4, 100, nb.NBODY_F64))[0]
    print("C3 100-step |dE/E|: F32C", d32, "FP64", d64, "ratio", d32 / d64)
    assert d32 <= 2 * d64, (d32, d64)


@pytest.mark.skipif(os.environ.get("NBODY_LONG") != "1", reason="13-minute run; NBODY_LONG=1")
def test_c3_full_1000_steps_drift_within_twice_fp64():
    n = 131072
    pos, vel, mass = ic.plummer(n, seed=3)
    drift = {}
    for mode in (nb.NBODY_F32C, nb.NBODY_F64):
        with nb.nbody_init(n, 1e-3, mode=mode, reorder_every=10) as ctx:
            p, v, m = dev(pos), dev(vel), dev(mass)
            acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
            pot = torch.empty(n, dtype=torch.float64, device="cuda")
            nb.nbody_forces(ctx, p, m, acc, pot)
            e0 = nb.nbody_energy(ctx, p, v, m, pot)[0]
            d = torch.empty((1000, 1, 9), dtype=torch.float64, device="cuda")
            nb.nbody_step(ctx, p, v, m, acc, pot, 1e-4, 1000, d)
            e = host(d)[:, 0, :]
            drift[mode] = (np.abs(e[:, 2] - e0[2]).max() / abs(e0[2]),
                           np.abs(e[:, 3:6] - e0[3:6]).max())
    assert drift[nb.NBODY_F32C][0] <= 2 * drift[nb.NBODY_F64][0], drift
    print("C3 drift", drift)


def test_c4_ensemble_all_clusters_match_oracle(oracle):
    ens = ic.ensemble(512, seed=4)
    n = ens.mass.shape[0]
    with nb.nbody_init(n, ens.eps, cluster_offsets=ens.offsets, reorder_every=1) as ctx:
        p, v, m = dev(ens.pos), dev(ens.vel), dev(ens.mass)
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, p, m, acc, pot)
        a, ph = host(acc), host(pot)
        worst = {"median": 0.0, "max": 0.0, "paper": 0.0, "paper_rms": 0.0}
        for c in range(512):
            b, e = ens.offsets[c], ens.offsets[c + 1]
            ra, rp = oracle.forces(ens.pos[:, b:e], ens.mass[b:e], ens.eps[c])
            s = check_f32c(a[:, b:e], ph[b:e], ra, rp, rms=False)
            if s["paper_rms"] > worst["paper_rms"]:
                own = np.linalg.norm(ra, axis=0)
                k = int(np.argmax(np.abs(a[:, b:e] - ra).max(axis=0)))
                worst["rms_worst"] = {"cluster": c, "n_c": int(e - b), "particle": k,
                                      "abs_a_over_rms": float(own[k] / np.sqrt(np.mean(own ** 2))),
                                      "rel_err": float(metrics.rel_acc_errors(a[:, b:e], ra)[k])}
            worst = {kk: (max(worst[kk], s[kk]) if kk in s else v) for kk, v in worst.items()}
        print("C4 accuracy, worst over 512 clusters:", worst)
        d = torch.empty((20, 512, 9), dtype=torch.float64, device="cuda")
        nb.nbody_step(ctx, p, v, m, acc, pot, 1e-3, 20, d)
        dg = host(d)
    # per-cluster momentum: FP32 pair terms break Newton's third law only at the
    # rounding level, so |dP| <= steps * dt * (max rel. error 1e-4) * sum m|a|
    assert np.all(np.isfinite(dg)) and np.all(dg[:, :, 2] < 0)
    for c in range(512):
        b, e = ens.offsets[c], ens.offsets[c + 1]
        bound = 20 * 1e-3 * 1e-4 * (ens.mass[b:e] * np.linalg.norm(a[:, b:e], axis=0)).sum()
        assert np.abs(dg[:, c, 3:6]).max() <= bound, c


def test_c4_drift_within_twice_fp64_every_cluster():
    # the batched form: 100 steps of all 512 clusters in one launch per step,
    # F32C and FP64 from the same state; every cluster's |dE/E| drift (its
    # own phi) within twice the FP64 path's, no floor
    ens = ic.ensemble(512, seed=4)
    d32 = drift(energy_track(ens.pos, ens.vel, ens.mass, ens.eps, 1e-3, 100, nb.NBODY_F32C,
                             offsets=ens.offsets))
    d64 = drift(energy_track(ens.pos, ens.vel, ens.mass, ens.eps, 1e-3, 100, nb.NBODY_F64,
                             offsets=ens.offsets))
    ratio = d32 / d64
    print("C4 100-step drift ratio per cluster: max", ratio.max(), "median", np.median(ratio))
    assert np.all(ratio <= 2), (np.argmax(ratio), ratio.max(), d32[np.argmax(ratio)],
                                d64[np.argmax(ratio)])


def test_c5_full_size_sampled_rows(oracle):
    pos, vel, mass = ic.two_plummer(524288, seed=5)
    n = mass.shape[0]
    with nb.nbody_init(n, 1e-3, reorder_every=1, flags=nb.NBODY_FLAG_AUTOTUNE) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, p, m, acc, pot)
        rows = ic.sample_rows(n, 1024, 77)
        ra, rp = oracle.forces_rows(pos, mass, 1e-3, rows)
        s = check_f32c(host(acc)[:, rows], host(pot)[rows], ra, rp)
        # with thousands of j-tiles per particle the cross-tile Kahan fold is
        # what keeps the medians low: plain FP32 folds give 2.9e-7 and 2.1e-7
        # here (measured with the ablation build), compensated ones 5e-8 and 8e-9
        assert s["median"] <= 1.5e-7 and s["pot_median"] <= 5e-8, s
        # one graph-replayed step, then the same check at the new positions
        nb.nbody_step(ctx, p, v, m, acc, pot, 1e-4, 1)
        ph = host(p)
        ra, rp = oracle.forces_rows(ph, mass, 1e-3, rows)
        check_f32c(host(acc)[:, rows], host(pot)[rows], ra, rp)


def test_paper_scale_jerk_full_size_sampled_rows(oracle):
    # the paper's N with the configuration bench.py's paper-scale section times
    # (default 512-wide j-tiles from 65 536 particles), rows against the oracle
    n = 102400
    pos, vel, mass = ic.plummer(n, seed=6)
    with nb.nbody_init(n, 1e-3, reorder_every=1) as ctx:
        assert nb.nbody_get_jerk_tiles(ctx) == (0, 0, 0, 0, 0)   # built on first use
        p, v, m = dev(pos), dev(vel), dev(mass)
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        jerk = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces_jerk(ctx, p, v, m, acc, jerk, pot)
        assert nb.nbody_get_jerk_tiles(ctx)[2] == 512
        rows = ic.sample_rows(n, 512, 78)
        ra, rj, rp = oracle.forces_jerk_rows(pos, vel, mass, 1e-3, rows)
        check_f32c(host(acc)[:, rows], host(pot)[rows], ra, rp)
        s = metrics.summary(host(jerk)[:, rows], rj)
        assert s["median"] <= 1e-5, s
        assert metrics.paper_metric(host(jerk)[:, rows], rj) <= 2e-3
        assert metrics.paper_metric_rms(host(jerk)[:, rows], rj) <= 2e-3


def test_block_steps_full_size_synchronised_state(oracle):
    # bench.py's block-step workload over its first dt_max: every particle
    # ends at t_end with a power-of-two step, and its stored acceleration and
    # jerk (taken at its last predicted state) agree with a fresh oracle
    # evaluation at the final state to the last correction's O(dt^4) plus the
    # F32C error
    n = 102400
    pos, vel, mass = ic.plummer(n, seed=7)
    dt_max, dt_min = 2.0 ** -7, 2.0 ** -22
    with nb.nbody_init(n, 1e-3, reorder_every=4) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        jerk = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_block_start(ctx, p, v, m, acc, jerk, pot, dt_max, dt_min, 0.02, 0.01)
        blocks, evals = nb.nbody_block_advance(ctx, p, v, m, acc, jerk, pot, dt_max)
        t, dt = nb.nbody_block_state(ctx)
    assert blocks > 10 and n <= evals < blocks * n
    assert np.all(t == dt_max)
    lg = np.log2(dt)
    assert np.all(lg == np.round(lg)) and dt.max() <= dt_max and dt.min() >= dt_min
    rows = ic.sample_rows(n, 256, 79)
    ra, rj, rp = oracle.forces_jerk_rows(host(p), host(v), mass, 1e-3, rows)
    s = metrics.summary(host(acc)[:, rows], ra)
    assert s["median"] <= 1e-6 and s["max"] <= 1e-4, s
    assert metrics.summary(host(jerk)[:, rows], rj)["median"] <= 1e-4


def test_measured_pipe_rates_are_plausible():
    from paper_2509_19294_gb300 import probe
    r = probe.measure_pipes()
    assert 32 <= r["fp32_lanes_per_clk_sm"] <= 260, r
    assert 4 <= r["mufu_rsqrt_per_clk_sm"] <= 64, r
    assert 1 <= r["pair_arith_pairs_per_clk_sm"] <= 20, r
    assert 0 < r["fp64_fma_per_clk_sm"] <= 64, r
