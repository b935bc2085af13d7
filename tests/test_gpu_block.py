"""Individual (block) time steps on the GPU against the oracle's block scheme (GPU).

The schedule is integer-like (power-of-two steps, an active set), decided from
FP64 quantities on both sides.  With NBODY_F64 forces the GPU takes the same
decisions as the oracle, so the steps, the number of block steps and of
evaluations match exactly and the trajectories to rounding.  With NBODY_F32C
forces a step decision can flip where the criterion sits on a power-of-two
boundary, so those runs are compared statistically and within the accuracy of
the integration.
"""
import numpy as np
import pytest
import torch

import paper_2509_19294_gb300 as nb
from paper_2509_19294_gb300 import ic
from tests import metrics
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu

DT_MAX, DT_MIN = 2.0 ** -6, 2.0 ** -20
T_END = 2.0 ** -4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_19294_gb300 import build
    build.build()
    nb.load()
    torch.cuda.init()


def block_run(pos, vel, mass, eps, mode, eta=0.02, eta_s=0.01, t_end=T_END, offsets=None, flags=0,
              jerk_tiles=None, dt_max=DT_MAX, dt_min=DT_MIN, **kw):
    n = mass.shape[0]
    with nb.nbody_init(n, eps, mode=mode, cluster_offsets=offsets, flags=flags, **kw) as ctx:
        if jerk_tiles is not None:
            nb.nbody_set_jerk_tiles(ctx, jerk_tiles)
        p, v, m = dev(pos), dev(vel), dev(mass)
        a = torch.empty((3, n), dtype=torch.float64, device="cuda")
        j = torch.empty((3, n), dtype=torch.float64, device="cuda")
        ph = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_block_start(ctx, p, v, m, a, j, ph, dt_max, dt_min, eta, eta_s)
        blocks, evals = nb.nbody_block_advance(ctx, p, v, m, a, j, ph, t_end)
        t, dt = nb.nbody_block_state(ctx)
        return host(p), host(v), host(a), host(j), dt, t, blocks, evals


def cluster_system(n=600, seed=51):
    pos, vel, mass = ic.plummer(n, seed=seed)
    return pos, vel, mass


def test_f64_block_steps_match_oracle_exactly(oracle):
    pos, vel, mass = cluster_system()
    gp, gv, ga, gj, gdt, gt, gb, ge = block_run(pos, vel, mass, 0.01, nb.NBODY_F64)
    rp, rv, ra, rj, _, rdt, rb, re = oracle.block_hermite(pos, vel, mass, 0.01, T_END, DT_MAX, DT_MIN,
                                                         0.02, 0.01)
    assert len(np.unique(rdt)) > 1            # the particles really take different steps
    assert np.array_equal(gdt, rdt) and gb == rb and ge == re
    assert np.all(gt == T_END)
    np.testing.assert_allclose(gp, rp, rtol=0, atol=1e-12)
    np.testing.assert_allclose(gv, rv, rtol=0, atol=1e-10)
    assert metrics.rel_acc_errors(ga, ra).max() <= 1e-10


@pytest.mark.parametrize("mode", [nb.NBODY_F64, nb.NBODY_F32C])
def test_equal_steps_reduce_to_shared_hermite(mode):
    pos, vel, mass = cluster_system(500, 52)
    n = 500
    gp, gv, ga, gj, gdt, _, gb, ge = block_run(pos, vel, mass, 0.01, mode, eta=1e30, eta_s=1e30)
    assert np.all(gdt == DT_MAX) and gb == 4 and ge == 4 * n
    with nb.nbody_init(n, 0.01, mode=mode) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        a = torch.empty((3, n), dtype=torch.float64, device="cuda")
        j = torch.empty((3, n), dtype=torch.float64, device="cuda")
        ph = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_forces_jerk(ctx, p, v, m, a, j, ph)
        nb.nbody_step_hermite(ctx, p, v, m, a, j, ph, DT_MAX, 4)
        sp, sv = host(p), host(v)
    if mode == nb.NBODY_F64:
        assert np.array_equal(gp, sp) and np.array_equal(gv, sv)
    else:
        # same scheme, FP32C forces on the subset path vs the full path: each
        # evaluation is within the F32C bound (max 1e-4, median 1e-6 relative),
        # so the two differ by at most twice that, propagated as
        # |dx| <= nsteps^2 dt^2 rel max|a| and |dv| <= nsteps dt rel max|a|
        amax = np.abs(ga).max()
        dx, dv = np.abs(gp - sp), np.abs(gv - sv)
        assert dx.max() <= 16 * DT_MAX ** 2 * 2e-4 * amax, dx.max()
        assert np.median(dx) <= 16 * DT_MAX ** 2 * 2e-6 * amax, np.median(dx)
        assert dv.max() <= 4 * DT_MAX * 2e-4 * amax, dv.max()
        assert np.median(dv) <= 4 * DT_MAX * 2e-6 * amax, np.median(dv)


# j-tile widths 128 (default at this N), 256 and 512: each has its own subset kernels
@pytest.mark.parametrize("jerk_tiles", [None, (128, 2, 256, 0, 2), (256, 2, 512, 0, 1)])
def test_f32c_block_steps_track_oracle(oracle, jerk_tiles):
    pos, vel, mass = cluster_system(2000, 53)
    gp, gv, ga, gj, gdt, gt, gb, ge = block_run(pos, vel, mass, 0.005, nb.NBODY_F32C,
                                                jerk_tiles=jerk_tiles)
    rp, rv, ra, rj, _, rdt, rb, re = oracle.block_hermite(pos, vel, mass, 0.005, T_END, DT_MAX, DT_MIN,
                                                         0.02, 0.01)
    assert np.all(gt == T_END)
    assert np.mean(gdt == rdt) >= 0.99
    assert abs(ge - re) <= 0.01 * re
    dx = np.abs(gp - rp).max(axis=0)
    assert np.median(dx) <= 1e-10 and dx.max() <= 1e-7, (np.median(dx), dx.max())
    s = metrics.summary(ga, ra)
    assert s["median"] <= 1e-6, s


def test_f32c_step_criterion_outside_the_float_range_takes_the_fp64_decision():
    # G x 2^40 with every time x 2^-20 (velocities x 2^20) is the same motion:
    # the acceleration and its first three derivatives scale by 2^40, 2^60,
    # 2^80 and 2^100, and every FP32 and FP64 operation before the step
    # criterion scales exactly by a power of two.  The squared norms then
    # leave the range (2^-120 .. 2^120) in which the F32C corrector takes the
    # criterion in FP32, so the scaled run takes the FP64 decisions: the
    # unscaled run's steps except where FP32 and FP64 rounding of the
    # criterion fall on either side of a power of two, the same evaluations
    # and, away from such flips, the same trajectories
    pos, vel, mass = cluster_system(2000, 53)
    s = 2.0 ** 20
    bp, bv, _, _, bdt, bt, bb, be = block_run(pos, vel, mass, 0.005, nb.NBODY_F32C)
    sp, sv, _, _, sdt, st, sb, se = block_run(pos, vel * s, mass, 0.005, nb.NBODY_F32C, G=s * s,
                                              t_end=T_END / s, dt_max=DT_MAX / s, dt_min=DT_MIN / s)
    assert np.all(st * s == T_END) and np.all(bt == T_END)
    same = sdt * s == bdt
    assert np.mean(same) >= 0.99, np.mean(same)
    assert abs(sb - bb) <= 0.01 * bb and abs(se - be) <= 0.01 * be, (sb, bb, se, be)
    dx = np.abs(sp - bp).max(axis=0)
    assert np.median(dx) <= 1e-10 and dx.max() <= 1e-7, (np.median(dx), dx.max())
    dv = np.abs(sv / s - bv).max(axis=0)
    assert np.median(dv) <= 1e-10 and dv.max() <= 1e-5, (np.median(dv), dv.max())


def test_f32c_block_trace_records_every_step():
    # NBODY_FLAG_TRACE: one record per step, each step's size its active
    # count; two advance calls, each read back after it
    pos, vel, mass = cluster_system(2000, 53)
    n = mass.shape[0]
    with nb.nbody_init(n, 0.005, mode=nb.NBODY_F32C, flags=nb.NBODY_FLAG_TRACE) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        a = torch.empty((3, n), dtype=torch.float64, device="cuda")
        j = torch.empty((3, n), dtype=torch.float64, device="cuda")
        ph = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_block_start(ctx, p, v, m, a, j, ph, DT_MAX, DT_MIN, 0.02, 0.01)
        b1, e1 = nb.nbody_block_advance(ctx, p, v, m, a, j, ph, T_END / 2)
        s1, n1 = nb.nbody_block_trace(ctx, 1, b1)
        b2, e2 = nb.nbody_block_advance(ctx, p, v, m, a, j, ph, T_END)
        s2, n2 = nb.nbody_block_trace(ctx, b1 + 1, b2)
        for secs, act, blocks, evals in ((s1, n1, b1, e1), (s2, n2, b2 - b1, e2 - e1)):
            assert len(secs) == blocks and len(act) == blocks
            assert np.all(act >= 1) and act.sum() == evals
            assert np.all(secs > 0) and secs.sum() < 10.0
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_block_trace(ctx, 1, b2 + 1)  # the record after the last one does not exist
        assert e.value.code == nb.NBODY_EINVAL
    with nb.nbody_init(n, 0.005, mode=nb.NBODY_F32C) as ctx:
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_block_trace(ctx, 1, 1)
        assert e.value.code == nb.NBODY_ESTATE


@pytest.mark.parametrize("mode", [nb.NBODY_F64, nb.NBODY_F32C])
def test_ensemble_block_steps_equal_independent_clusters(oracle, mode):
    ens = ic.ensemble(5, seed=54, n_min=256, n_max=900)
    gp, gv, ga, gj, gdt, gt, gb, ge = block_run(ens.pos, ens.vel, ens.mass, ens.eps, mode,
                                                offsets=ens.offsets)
    total = 0
    for c in range(5):
        b, e = ens.offsets[c], ens.offsets[c + 1]
        rp, rv, ra, rj, _, rdt, rb, re = oracle.block_hermite(
            ens.pos[:, b:e], ens.vel[:, b:e], ens.mass[b:e], ens.eps[c], T_END, DT_MAX, DT_MIN, 0.02,
            0.01)
        total += re
        if mode == nb.NBODY_F64:
            assert np.array_equal(gdt[b:e], rdt)
            np.testing.assert_allclose(gp[:, b:e], rp, rtol=0, atol=1e-12)
        else:
            assert np.mean(gdt[b:e] == rdt) >= 0.98
            assert np.abs(gp[:, b:e] - rp).max() <= 1e-7
    if mode == nb.NBODY_F64:
        assert ge == total


@pytest.mark.parametrize("mode", [nb.NBODY_F64, nb.NBODY_F32C])
def test_block_steps_with_an_empty_cluster(oracle, mode):
    p1, v1, m1 = ic.plummer(300, seed=59)
    p2, v2, m2 = ic.plummer(400, seed=60)
    pos, vel, mass = np.hstack([p1, p2]), np.hstack([v1, v2]), np.concatenate([m1, m2])
    offsets = np.array([0, 300, 300, 700])
    gp, gv, ga, gj, gdt, gt, gb, ge = block_run(pos, vel, mass, np.array([0.01, 0.02, 0.01]), mode,
                                                offsets=offsets)
    assert np.all(gt == T_END)
    for (b, e), (pp, vv, mm) in zip([(0, 300), (300, 700)], [(p1, v1, m1), (p2, v2, m2)]):
        rp, rv, ra, rj, _, rdt, rb, re = oracle.block_hermite(pp, vv, mm, 0.01, T_END, DT_MAX, DT_MIN,
                                                             0.02, 0.01)
        if mode == nb.NBODY_F64:
            assert np.array_equal(gdt[b:e], rdt)
            np.testing.assert_allclose(gp[:, b:e], rp, rtol=0, atol=1e-12)
        else:
            assert np.mean(gdt[b:e] == rdt) >= 0.98
            assert np.abs(gp[:, b:e] - rp).max() <= 1e-7


@pytest.mark.parametrize("mode", [nb.NBODY_F64, nb.NBODY_F32C])
def test_block_graph_equals_eager(mode):
    pos, vel, mass = cluster_system(700, 55)
    g = block_run(pos, vel, mass, 0.01, mode, reorder_every=5)
    e = block_run(pos, vel, mass, 0.01, mode, reorder_every=5, flags=nb.NBODY_FLAG_NO_GRAPH)
    for x, y in zip(g, e):
        assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("mode", [nb.NBODY_F64, nb.NBODY_F32C])
def test_block_steps_without_softening(oracle, mode):
    # eps = 0: the EPS_ZERO kernel variants (and the few-particle path's
    # r^2 > 0 guard); a loose cluster so that no pair comes too close
    pos, vel, mass = ic.plummer(400, seed=58)
    pos = pos * 4.0
    vel = vel / 2.0
    gp, gv, ga, gj, gdt, gt, gb, ge = block_run(pos, vel, mass, 0.0, mode)
    rp, rv, ra, rj, _, rdt, rb, re = oracle.block_hermite(pos, vel, mass, 0.0, T_END, DT_MAX, DT_MIN,
                                                         0.02, 0.01)
    assert len(np.unique(rdt)) > 1
    if mode == nb.NBODY_F64:
        assert np.array_equal(gdt, rdt) and gb == rb and ge == re
        np.testing.assert_allclose(gp, rp, rtol=0, atol=1e-12)
    else:
        assert np.mean(gdt == rdt) >= 0.98
        assert np.abs(gp - rp).max() <= 1e-7
        assert metrics.summary(ga, ra)["median"] <= 1e-6


def wide_tile_binary(n_field=30, seed=61, sep=1e-3, where=8.0):
    """A loose field of n_field stars (one centre tile of extent ~10) and a
    circular binary of separation sep placed `where` from the centre: its
    members' FP32 offsets from the tile centre are ~where, so rounding them
    once (u * where ~ 5e-7) would be a relative error ~5e-4 of their
    separation."""
    pos, vel, _ = ic.plummer(n_field, seed=seed)
    pos, vel = pos * 5.0, vel / np.sqrt(5.0)
    n = n_field + 2
    mass = np.full(n, 1.0 / n)
    v = np.sqrt(2.0 * mass[0] / sep) / 2.0  # each member's speed on the circular orbit
    bp = np.array([[where - sep / 2, where + sep / 2], [0.0, 0.0], [0.0, 0.0]])
    bv = np.array([[0.0, 0.0], [-v, v], [0.0, 0.0]])
    return np.hstack([pos, bp]), np.hstack([vel, bv]), mass


def test_f32c_few_particle_pass_differences_close_pairs_exactly(oracle):
    # <= 32 particles: every block step runs the few-particle pass.  The
    # binary takes the smallest steps; its orbit (~20 periods) and its members'
    # accelerations follow the oracle to the FP32 accuracy of the pair terms,
    # not to that of the offsets' magnitude.
    pos, vel, mass = wide_tile_binary()
    t_end = DT_MAX
    gp, gv, ga, gj, gdt, gt, gb, ge = block_run(pos, vel, mass, 1e-4, nb.NBODY_F32C, t_end=t_end)
    rp, rv, ra, rj, _, rdt, rb, re = oracle.block_hermite(pos, vel, mass, 1e-4, t_end, DT_MAX, DT_MIN,
                                                         0.02, 0.01)
    assert rdt[-1] <= 2.0 ** -14 and rdt[-1] < rdt[:-2].min()  # the binary takes the smallest steps
    # offsets rounded to FP32 once (error ~5e-4 of the separation) make the
    # binary's forces noisy enough for the step criterion (its third
    # derivative estimate scales as da / h^3) to shrink the step towards
    # dt_min, multiplying the block steps; differenced exactly, the binary
    # keeps the oracle's step and the run its schedule
    assert np.array_equal(gdt[-2:], rdt[-2:]) and abs(gb - rb) <= 0.05 * rb, (gb, rb)
    assert np.abs(gp[:, :-2] - rp[:, :-2]).max() <= 1e-10
    assert np.abs(gp[:, -2:] - rp[:, -2:]).max() <= 5e-7  # ~20 orbits of FP32 pair arithmetic
    assert metrics.rel_acc_errors(ga[:, -2:], ra[:, -2:]).max() <= 2e-4


def block_run_chunked(pos, vel, mass, eps, mode, t_ends, shift=None, **kw):
    """block_run advancing through t_ends in turn; shift (a 3-vector) is added
    to every position on the device after the first advance call."""
    n = mass.shape[0]
    with nb.nbody_init(n, eps, mode=mode, **kw) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        a = torch.empty((3, n), dtype=torch.float64, device="cuda")
        j = torch.empty((3, n), dtype=torch.float64, device="cuda")
        ph = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_block_start(ctx, p, v, m, a, j, ph, DT_MAX, DT_MIN, 0.02, 0.01)
        for k, te in enumerate(t_ends):
            blocks, evals = nb.nbody_block_advance(ctx, p, v, m, a, j, ph, te)
            if k == 0 and shift is not None:
                p += torch.tensor(shift, dtype=torch.float64, device="cuda").reshape(3, 1)
        t, dt = nb.nbody_block_state(ctx)
        return host(p), host(v), host(a), host(j), dt, t, blocks, evals


@pytest.mark.parametrize("mode", [nb.NBODY_F64, nb.NBODY_F32C])
def test_block_steps_in_chunks_with_resorts_track_oracle(oracle, mode):
    # four advance calls (each F32C one starts from the rows again) and a
    # Morton re-sort at every dt_max (a fresh F32C pack of new tile frames)
    pos, vel, mass = cluster_system(1500, 62)
    t_ends = [DT_MAX * k for k in (1, 2, 3, 4)]
    gp, gv, ga, gj, gdt, gt, gb, ge = block_run_chunked(pos, vel, mass, 0.005, mode, t_ends,
                                                        reorder_every=1)
    rp, rv, ra, rj, _, rdt, rb, re = oracle.block_hermite(pos, vel, mass, 0.005, T_END, DT_MAX, DT_MIN,
                                                         0.02, 0.01)
    assert np.all(gt == T_END)
    if mode == nb.NBODY_F64:
        assert np.array_equal(gdt, rdt) and gb == rb and ge == re
        np.testing.assert_allclose(gp, rp, rtol=0, atol=1e-12)
    else:
        assert np.mean(gdt == rdt) >= 0.99 and abs(ge - re) <= 0.01 * re
        dx = np.abs(gp - rp).max(axis=0)
        assert np.median(dx) <= 1e-10 and dx.max() <= 1e-7, (np.median(dx), dx.max())


@pytest.mark.parametrize("mode", [nb.NBODY_F64, nb.NBODY_F32C])
def test_block_advance_reads_the_callers_arrays_again(mode):
    # the caller translates every particle between two advance calls; forces
    # are translation invariant, so the run is the untranslated one moved by
    # the same vector (state kept from the previous call would ignore it)
    pos, vel, mass = cluster_system(800, 63)
    d = np.array([0.25, -0.5, 0.125])
    t_ends = [DT_MAX * 2, T_END]
    gp0, *_, gb0, ge0 = block_run_chunked(pos, vel, mass, 0.01, mode, t_ends)
    gp1, *_, gb1, ge1 = block_run_chunked(pos, vel, mass, 0.01, mode, t_ends, shift=d)
    dx = np.abs(gp1 - d[:, None] - gp0).max(axis=0)
    if mode == nb.NBODY_F64:
        assert dx.max() <= 1e-10, dx.max()
    else:  # different tile centres round the offsets differently
        assert np.median(dx) <= 1e-9 and dx.max() <= 1e-6, (np.median(dx), dx.max())
    assert abs(gb1 - gb0) <= 0.01 * gb0 and abs(ge1 - ge0) <= 0.01 * ge0


def tiny_system(n, seed=64):
    if n == 1:
        return np.zeros((3, 1)), np.array([[0.1], [-0.2], [0.05]]), np.ones(1)
    if n == 2:  # a circular binary
        pos = np.array([[-0.5, 0.5], [0.0, 0.0], [0.0, 0.0]])
        vel = np.array([[0.0, 0.0], [-0.5, 0.5], [0.0, 0.0]])
        return pos, vel, np.full(2, 0.5)
    return ic.plummer(n, seed=seed)


@pytest.mark.parametrize("mode", [nb.NBODY_F64, nb.NBODY_F32C])
@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 129])
def test_block_steps_tiny_systems(oracle, mode, n):
    # one particle (no force: every step dt_max), a binary, and active sets on
    # both sides of the few-particle limit (32) and of one 128-slot tile
    pos, vel, mass = tiny_system(n)
    gp, gv, ga, gj, gdt, gt, gb, ge = block_run(pos, vel, mass, 0.01, mode)
    rp, rv, ra, rj, _, rdt, rb, re = oracle.block_hermite(pos, vel, mass, 0.01, T_END, DT_MAX, DT_MIN,
                                                         0.02, 0.01)
    assert np.all(gt == T_END)
    if n == 1:
        assert np.all(gdt == DT_MAX) and np.all(ga == 0.0) and np.all(gj == 0.0)
    if mode == nb.NBODY_F64:
        assert np.array_equal(gdt, rdt) and gb == rb and ge == re
        np.testing.assert_allclose(gp, rp, rtol=0, atol=1e-12)
    else:
        assert np.mean(gdt == rdt) >= 0.95
        assert np.abs(gp - rp).max() <= 1e-7


def test_block_steps_save_evaluations():
    pos, vel, mass = cluster_system(3000, 56)
    *_, gb, ge = block_run(pos, vel, mass, 0.002, nb.NBODY_F32C)
    # a shared step at the smallest block step would cost n * blocks evaluations
    assert ge < 0.5 * 3000 * gb


def test_block_api_errors():
    n = 64
    pos, vel, mass = cluster_system(n, 57)
    with nb.nbody_init(n, 0.01) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        a = torch.empty((3, n), dtype=torch.float64, device="cuda")
        j = torch.empty((3, n), dtype=torch.float64, device="cuda")
        with pytest.raises(nb.NBodyError):
            nb.nbody_block_advance(ctx, p, v, m, a, j, None, T_END)
    with nb.nbody_init(n, 0.01) as ctx:
        with pytest.raises(nb.NBodyError):
            nb.nbody_block_start(ctx, pos, vel, mass, np.empty((3, n)), np.empty((3, n)), None,
                                 DT_MAX, DT_MIN, 0.02, 0.01)
    with nb.nbody_init(n, 0.01) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        a = torch.empty((3, n), dtype=torch.float64, device="cuda")
        j = torch.empty((3, n), dtype=torch.float64, device="cuda")
        with pytest.raises(nb.NBodyError):
            nb.nbody_block_start(ctx, p, v, m, a, j, None, 0.03, DT_MIN, 0.02, 0.01)
    with nb.nbody_init(n, 0.01) as ctx:   # errors are sticky: a fresh context
        p, v, m = dev(pos), dev(vel), dev(mass)
        a = torch.empty((3, n), dtype=torch.float64, device="cuda")
        j = torch.empty((3, n), dtype=torch.float64, device="cuda")
        nb.nbody_block_start(ctx, p, v, m, a, j, None, DT_MAX, DT_MIN, 0.02, 0.01)
        with pytest.raises(nb.NBodyError):
            nb.nbody_block_advance(ctx, p, v, m, a, j, None, DT_MAX * 1.5)
    for mode, ok in ((nb.NBODY_F32C, False), (nb.NBODY_F64, True)):
        # F32C block steps keep step lengths as floats: dt_min >= 2^-126
        with nb.nbody_init(n, 0.01, mode=mode) as ctx:
            p, v, m = dev(pos), dev(vel), dev(mass)
            a = torch.empty((3, n), dtype=torch.float64, device="cuda")
            j = torch.empty((3, n), dtype=torch.float64, device="cuda")
            if ok:
                nb.nbody_block_start(ctx, p, v, m, a, j, None, 2.0 ** -100, 2.0 ** -130, 0.02, 0.01)
            else:
                with pytest.raises(nb.NBodyError):
                    nb.nbody_block_start(ctx, p, v, m, a, j, None, 2.0 ** -100, 2.0 ** -130, 0.02, 0.01)


@pytest.mark.parametrize("n", [24, 200])
def test_f32c_block_potential_has_no_self_term(oracle, n):
    # a heavy particle (m = 1) among light ones with eps = 1e-6: its self term
    # m / eps is ~1e10 times its potential.  One block step with every particle
    # active (the few-particle pass for n = 24, the subset kernel for n = 200):
    # the stored potential equals the oracle's block scheme to the FP32C bound
    rng = np.random.default_rng(71 + n)
    pos = rng.uniform(-0.5, 0.5, size=(3, n))
    vel = np.zeros((3, n))
    mass = np.full(n, 1e-6)
    h = n // 3
    mass[h] = 1.0
    with nb.nbody_init(n, 1e-6, mode=nb.NBODY_F32C) as ctx:
        p, v, m = dev(pos), dev(vel), dev(mass)
        a = torch.empty((3, n), dtype=torch.float64, device="cuda")
        j = torch.empty((3, n), dtype=torch.float64, device="cuda")
        ph = torch.empty(n, dtype=torch.float64, device="cuda")
        nb.nbody_block_start(ctx, p, v, m, a, j, ph, 2.0 ** -10, 2.0 ** -30, 0.02, 0.01)
        _, rj, rp0 = oracle.forces_jerk(pos, vel, mass, 1e-6)
        ep = metrics.rel_pot_errors(host(ph), rp0)
        assert ep[h] <= 1e-5 and ep.max() <= 1e-4, (ep[h], ep.max())
        blocks, evals = nb.nbody_block_advance(ctx, p, v, m, a, j, ph, 2.0 ** -10)
        gpot = host(ph)
    *_, rpot, rdt, rb, re = oracle.block_hermite(pos, vel, mass, 1e-6, 2.0 ** -10, 2.0 ** -10,
                                                 2.0 ** -30, 0.02, 0.01)
    assert (blocks, evals) == (rb, re) == (1, n)
    ep = metrics.rel_pot_errors(gpot, rpot)
    assert ep[h] <= 1e-5 and ep.max() <= 1e-4, (ep[h], ep.max())
