"""Parity of the CUDA path with the FP64 oracle (GPU).

Tolerances:
  * NBODY_F64 against the oracle: per-particle relative acceleration error
    <= 1e-12 (both are FP64 sums of the same terms in different orders).
  * NBODY_F32C against the oracle: median relative acceleration error <= 1e-6
    and max <= 1e-4, potential median <= 1e-6 and max <= 1e-4, and the paper's
    own validation bound (Sec. 3: each component within 0.05 % of an undefined
    typical force magnitude), read against the particle's own |a_i| and, on
    the reference workloads (C2 here), also against the RMS |a| of the system.
"""
import numpy as np
import pytest
import torch

import paper_2509_19294_gb300 as nb
from paper_2509_19294_gb300 import ic
from tests import metrics
from tests.gpu_util import dev, forces, host

pytestmark = pytest.mark.gpu

F32C_MEDIAN = 1e-6
F32C_MAX = 1e-4
PAPER_BOUND = 5e-4


def assert_f32c(a, p, ra, rp):
    s = metrics.summary(a, ra, p, rp)
    assert s["median"] <= F32C_MEDIAN, s
    assert s["max"] <= F32C_MAX, s
    assert s["paper"] <= PAPER_BOUND, s
    assert s["pot_median"] <= F32C_MEDIAN, s
    assert s["pot_max"] <= F32C_MAX, s
    return s


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_19294_gb300 import build
    build.build()
    nb.load()
    torch.cuda.init()


def test_f64_plummer_1024_matches_oracle(oracle):
    pos, vel, mass = ic.plummer(1024, seed=1)
    a, p = forces(pos, mass, 0.01, mode=nb.NBODY_F64)
    ra, rp = oracle.forces(pos, mass, 0.01)
    assert metrics.rel_acc_errors(a, ra).max() <= 1e-12
    assert metrics.rel_pot_errors(p, rp).max() <= 1e-12


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_f32c_16384_log_uniform_masses(oracle, dist):
    n = 16384
    m = ic.log_uniform_masses(n, seed=2)
    if dist == "uniform":
        pos, _, mass = ic.uniform_sphere(n, seed=2, masses=m)
    else:
        pos, _, mass = ic.plummer(n, seed=2, masses=m)
    ra, rp = oracle.forces(pos, mass, 0.005)
    a, p = forces(pos, mass, 0.005)
    s = assert_f32c(a, p, ra, rp)
    assert s["paper_rms"] <= PAPER_BOUND, s          # against the RMS |a| too
    a64, p64 = forces(pos, mass, 0.005, mode=nb.NBODY_F64)
    assert metrics.rel_acc_errors(a64, ra).max() <= 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 255, 257, 1023, 4097])
@pytest.mark.parametrize("eps", [0.0, 0.01])
@pytest.mark.parametrize("mode", [nb.NBODY_F32C, nb.NBODY_F64])
def test_small_and_ragged_sizes(oracle, n, eps, mode):
    rng = np.random.default_rng(n)
    pos = rng.normal(size=(3, n))
    mass = rng.uniform(0.5, 1.5, n) / n
    a, p = forces(pos, mass, eps, mode=mode)
    ra, rp = oracle.forces(pos, mass, eps)
    if n == 1:
        assert np.all(a == 0.0) and np.all(p == 0.0)
        return
    if mode == nb.NBODY_F64:
        assert metrics.rel_acc_errors(a, ra).max() <= 1e-12
        assert metrics.rel_pot_errors(p, rp).max() <= 1e-12
    else:
        assert metrics.rel_acc_errors(a, ra).max() <= F32C_MAX
        assert metrics.rel_pot_errors(p, rp).max() <= F32C_MAX


def test_brute_force_tiny_systems(oracle):
    # N <= 8 on exactly representable coordinates: the regular configurations
    # of the oracle pins, now through the GPU path
    cube = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1],
                     [1, 1, 1]], np.float64).T
    for n in range(2, 9):
        pos = cube[:, :n].copy()
        mass = np.linspace(0.5, 2.0, n)
        for mode in (nb.NBODY_F32C, nb.NBODY_F64):
            a, p = forces(pos, mass, 0.0, mode=mode)
            ra, rp = oracle.forces(pos, mass, 0.0)
            tol = 1e-12 if mode == nb.NBODY_F64 else 1e-6
            np.testing.assert_allclose(a, ra, rtol=tol, atol=tol * np.abs(ra).max())
            np.testing.assert_allclose(p, rp, rtol=tol)


def test_coincident_particles_with_zero_softening(oracle):
    pos = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    mass = np.array([1.0, 2.0, 3.0])
    for mode in (nb.NBODY_F32C, nb.NBODY_F64):
        a, p = forces(pos, mass, 0.0, mode=mode)
        ra, rp = oracle.forces(pos, mass, 0.0)
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
        np.testing.assert_allclose(a, ra, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(p, rp, rtol=1e-6)


def test_every_tile_shape_and_split(oracle):
    n = 3001
    pos, _, mass = ic.plummer(n, seed=7)
    ra, rp = oracle.forces(pos, mass, 0.01)
    for block, p_, tj, minb in nb.nbody_tiles_supported():
        for split in (1, 3):
            a, p = forces(pos, mass, 0.01, tiles=(block, p_, tj, split, minb))
            s = metrics.summary(a, ra, p, rp)
            assert s["median"] <= F32C_MEDIAN and s["max"] <= F32C_MAX, (block, p_, tj, minb, split, s)


def test_translation_invariance_of_f32c(oracle):
    # tile-relative FP32 offsets keep every digit of close pairs far from the origin
    n = 8192
    pos, _, mass = ic.plummer(n, seed=8)
    ra, rp = oracle.forces(pos, mass, 0.005)
    shifted = pos + np.array([[1e3], [-1e3], [1e3]])
    a, p = forces(shifted, mass, 0.005)
    s = metrics.summary(a, ra, p, rp)
    assert s["median"] <= F32C_MEDIAN and s["max"] <= F32C_MAX, s


def test_gravitational_constant_scales(oracle):
    pos, _, mass = ic.plummer(2048, seed=9)
    a1, p1 = forces(pos, mass, 0.01, G=1.0)
    a2, p2 = forces(pos, mass, 0.01, G=2.5)
    np.testing.assert_allclose(a2, 2.5 * a1, rtol=1e-15)
    np.testing.assert_allclose(p2, 2.5 * p1, rtol=1e-15)


def test_bitwise_determinism():
    pos, _, mass = ic.plummer(20000, seed=10)
    a1, p1 = forces(pos, mass, 0.001, tiles=(128, 4, 256, 5))
    a2, p2 = forces(pos, mass, 0.001, tiles=(128, 4, 256, 5))
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)


def test_morton_reordering_keeps_results(oracle):
    n = 16384
    pos, _, mass = ic.plummer(n, seed=11)
    ra, rp = oracle.forces(pos, mass, 0.001)
    a, p = forces(pos, mass, 0.001, reorder_every=1)
    s = assert_f32c(a, p, ra, rp)
    a2, p2 = forces(pos, mass, 0.001, reorder_every=1)
    assert np.array_equal(a, a2) and np.array_equal(p, p2)


def test_host_arrays_are_staged(oracle):
    n = 5000
    pos, _, mass = ic.plummer(n, seed=12)
    acc_h = np.empty((3, n))
    pot_h = np.empty(n)
    with nb.nbody_init(n, 0.01) as ctx:
        nb.nbody_forces(ctx, pos, mass, acc_h, pot_h)
    a, p = forces(pos, mass, 0.01)
    assert np.array_equal(acc_h, a) and np.array_equal(pot_h, p)


def test_ensemble_matches_per_cluster_oracle(oracle):
    ens = ic.ensemble(12, seed=4, n_min=256, n_max=2048)
    for mode in (nb.NBODY_F32C, nb.NBODY_F64):
        a, p = forces(ens.pos, ens.mass, ens.eps, mode=mode, offsets=ens.offsets)
        for c in range(len(ens.eps)):
            b, e = ens.offsets[c], ens.offsets[c + 1]
            ra, rp = oracle.forces(ens.pos[:, b:e], ens.mass[b:e], ens.eps[c])
            if mode == nb.NBODY_F64:
                assert metrics.rel_acc_errors(a[:, b:e], ra).max() <= 1e-12
            else:
                s = metrics.summary(a[:, b:e], ra, p[b:e], rp)
                assert s["median"] <= F32C_MEDIAN and s["max"] <= F32C_MAX, (c, s)


def test_empty_clusters_and_empty_system():
    with nb.nbody_init(0, 0.1) as ctx:
        e = torch.empty((3, 0), dtype=torch.float64, device="cuda")
        m = torch.empty(0, dtype=torch.float64, device="cuda")
        nb.nbody_forces(ctx, e, m, e.clone(), m.clone())
        nb.nbody_step(ctx, e, e.clone(), m, e.clone(), m.clone(), 1e-3, 3)
        assert np.all(nb.nbody_energy(ctx, e, e.clone(), m, m.clone()) == 0.0)
    ens = ic.ensemble(3, seed=5, n_min=300, n_max=400)
    offs = np.array([0, 0, ens.offsets[1], ens.offsets[1], ens.offsets[2], ens.offsets[3]])
    eps = np.array([0.1, ens.eps[0], 0.1, ens.eps[1], ens.eps[2]])
    a, p = forces(ens.pos, ens.mass, eps, offsets=offs)
    a2, p2 = forces(ens.pos, ens.mass, ens.eps, offsets=ens.offsets)
    assert np.array_equal(a, a2) and np.array_equal(p, p2)


def test_invalid_arguments_set_sticky_error():
    n = 64
    pos, _, mass = ic.plummer(n, seed=13)
    with nb.nbody_init(n, 0.01) as ctx:
        lib = nb.load()
        rc = lib.nbody_forces(ctx.handle, None, None, None, None, None)
        assert rc == nb.NBODY_EINVAL
        rc = lib.nbody_forces(ctx.handle, dev(pos).data_ptr(), dev(mass).data_ptr(), 8, None, None)
        assert rc == nb.NBODY_ESTATE
        assert "NULL" in lib.nbody_last_error_message(ctx.handle).decode()


def test_check_finite_flag_reports_nan_input():
    n = 300
    pos, _, mass = ic.plummer(n, seed=14)
    pos[0, 17] = np.nan
    with nb.nbody_init(n, 0.01, flags=nb.NBODY_FLAG_CHECK_FINITE) as ctx:
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_forces(ctx, dev(pos), dev(mass), acc)
        assert e.value.code == nb.NBODY_ENONFINITE


def test_energy_matches_oracle(oracle):
    ens = ic.ensemble(5, seed=6, n_min=500, n_max=3000)
    _, rp_all = None, np.empty(ens.mass.shape[0])
    for c in range(5):
        b, e = ens.offsets[c], ens.offsets[c + 1]
        _, rp_all[b:e] = oracle.forces(ens.pos[:, b:e], ens.mass[b:e], ens.eps[c])
    with nb.nbody_init(ens.mass.shape[0], ens.eps, cluster_offsets=ens.offsets) as ctx:
        out = nb.nbody_energy(ctx, dev(ens.pos), dev(ens.vel), dev(ens.mass), dev(rp_all))
    for c in range(5):
        b, e = ens.offsets[c], ens.offsets[c + 1]
        want = oracle.energy(ens.pos[:, b:e], ens.vel[:, b:e], ens.mass[b:e], rp_all[b:e])
        np.testing.assert_allclose(out[c], want, rtol=1e-12, atol=1e-14)


def test_profile_counts_force_launches():
    n = 4096
    pos, _, mass = ic.plummer(n, seed=15)
    with nb.nbody_init(n, 0.01, flags=nb.NBODY_FLAG_PROFILE) as ctx:
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        p, m = dev(pos), dev(mass)
        for _ in range(5):
            nb.nbody_forces(ctx, p, m, acc)
        ms, cnt = nb.nbody_profile_read(ctx, reset=True)
        assert cnt == 5 and ms > 0.0
        assert nb.nbody_kernel_launches(ctx) >= 10


def test_reorder_paths_give_the_same_order():
    # a context whose largest cluster exceeds the shared-memory sort limit takes
    # the global bitonic path; a cluster's own results do not depend on the other
    # clusters, so they must equal (bitwise) those of a context that holds only
    # that cluster and takes the per-cluster shared-memory path
    big = ic.plummer(20000, seed=31)
    small = ic.plummer(3000, seed=32)
    pos = np.concatenate([big[0], small[0]], axis=1)
    mass = np.concatenate([big[2], small[2]])
    offs = np.array([0, 20000, 23000])
    tiles = (128, 2, 256, 1, 4)
    a1, p1 = forces(pos, mass, [0.002, 0.004], offsets=offs, tiles=tiles, reorder_every=1)
    a2, p2 = forces(small[0], small[2], 0.004, tiles=tiles, reorder_every=1)
    assert np.array_equal(a1[:, 20000:], a2) and np.array_equal(p1[20000:], p2)
    a3, p3 = forces(big[0], big[2], 0.002, tiles=tiles, reorder_every=1)
    assert np.array_equal(a1[:, :20000], a3) and np.array_equal(p1[:20000], p3)


def _heavy_system(n, seed):
    # one heavy particle among light ones, softening 1e-6: the heavy
    # particle's self term m_i / eps = 1e6 is ~1e10 times its true potential
    # (~1e-4); a self pair that entered the FP32 tile sums (and were removed
    # afterwards) would leave nothing of it
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.5, 0.5, size=(3, n))
    mass = np.full(n, 1e-6)
    mass[n // 3] = 1.0
    return pos, rng.normal(size=(3, n)) * 0.1, mass, n // 3


@pytest.mark.parametrize("n", [24, 300, 3001])
def test_self_pair_left_out_of_the_fp32_sums(oracle, n):
    pos, vel, mass, h = _heavy_system(n, 61 + n)
    ra, rj, rp = oracle.forces_jerk(pos, vel, mass, 1e-6)
    a, p = forces(pos, mass, 1e-6)
    ep = metrics.rel_pot_errors(p, rp)
    assert ep[h] <= 1e-5 and np.median(ep) <= 1e-6 and ep.max() <= 1e-4, (ep[h], ep.max())
    assert metrics.rel_acc_errors(a, ra).max() <= 1e-4
    with nb.nbody_init(n, 1e-6) as ctx:
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
        jerk = torch.empty((3, n), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces_jerk(ctx, dev(pos), dev(vel), dev(mass), acc, jerk, pot)
        ep = metrics.rel_pot_errors(host(pot), rp)
    assert ep[h] <= 1e-5 and ep.max() <= 1e-4, (ep[h], ep.max())
