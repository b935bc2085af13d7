// block_common.cuh -- device helpers shared by the block-step kernels
// (block_sched.cu, block_force.cu): the Hermite corrector, the step choice and
// the epilogue of an active particle.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "forces_f32c.cuh"
#include "nbody_internal.h"

namespace nbody {

// Grid for a grid-stride loop over `work` items (capped; the loops cover the rest).
inline int grid_of(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}


// 1/h, exact for a power of two h (built from its exponent; FP64 division is
// slow on this part), else the division.
__device__ __forceinline__ double recip_pow2(double h) {
    const long long b = __double_as_longlong(h);
    if ((b & 0x000FFFFFFFFFFFFFLL) == 0 && b > 0 && b < 0x7FE0000000000000LL)
        return __longlong_as_double(0x7FE0000000000000LL - b);
    return 1.0 / h;
}

// Next step of particle i after a step h, by Aarseth's criterion from the
// norms of the acceleration and its first three derivatives at the end of the
// step: halved while above it (not below dt_min), doubled once when allowed
// (<= dt_max, <= the criterion, and t_next a multiple of the doubled step --
// an integer test in units of dt_min).
__device__ __forceinline__ double criterion_step(const BlockCorrect &c, double h, double na, double nj,
                                                 double n2, double n3, long long tnq) {
    const double den = nj * n3 + n2 * n2;
    double nd = h;
    bool grow;
    if (den > 0.0 && c.dt_min >= 0x1p-500 && c.dt_max <= 0x1p500) {  // every p^2 below is exact
        // y = da^2 before its square root.  The criterion is only compared
        // with powers of two p, and for those p > sqrt_rn(y) <=> y < p^2
        // exactly (p^2 is exact, and no double lies within the half ulp below
        // p^2 that rounds up to p), so the square root is never taken
        const double y = c.eta * (na * n2 + nj * nj) / den;
        while (y < nd * nd && nd > c.dt_min) nd *= 0.5;
        grow = y >= 4.0 * h * h;
    } else {
        const double da = den > 0.0 ? sqrt(c.eta * (na * n2 + nj * nj) / den) : c.dt_max;
        while (nd > da && nd > c.dt_min) nd *= 0.5;
        grow = da >= 2.0 * h;
    }
    const long long q2 = (long long)(2.0 * h * recip_pow2(c.dt_min));  // 2h in units of dt_min
    if (nd == h && grow && 2.0 * h <= c.dt_max && (tnq & (q2 - 1)) == 0) nd = 2.0 * h;
    return nd;
}

// The same decision in FP32 from the squared norms (F32C path).  The criterion
// only selects a power of two, and its inputs carry the FP32 pair sums' error
// (~1e-7 relative), so FP32 rounding of its arithmetic (6e-8) decides nothing
// those inputs had not; a step waits on this chain, and FP32 square roots and
// divisions take a fraction of the FP64 ones' latency on this part.  Outside
// the range where every square, product and p^2 below is a normal float (and
// for NaN or infinite norms) it falls back to the FP64 decision.
__device__ __forceinline__ bool f32_criterion_range(double s) {
    return s == 0.0 || (s >= 0x1p-120 && s <= 0x1p120);
}

__device__ __forceinline__ double criterion_step_f32(const BlockCorrect &c, double h, double sa, double sj,
                                                     double s2, double s3, long long tnq) {
    if (!(f32_criterion_range(sa) && f32_criterion_range(sj) && f32_criterion_range(s2) &&
          f32_criterion_range(s3) && c.dt_min >= 0x1p-60 && c.dt_max <= 0x1p60))
        return criterion_step(c, h, sqrt(sa), sqrt(sj), sqrt(s2), sqrt(s3), tnq);
    const float na = sqrtf((float)sa), nj = sqrtf((float)sj), n2 = sqrtf((float)s2), n3 = sqrtf((float)s3);
    const float den = nj * n3 + n2 * n2;
    const float hf = (float)h, dmin = (float)c.dt_min;  // powers of two: exact
    float nd = hf;
    bool grow;
    if (den > 0.0f) {  // y < p^2 <=> p > sqrt(y) for a power of two p, as in FP64
        const float y = (float)c.eta * (na * n2 + nj * nj) / den;
        while (y < nd * nd && nd > dmin) nd *= 0.5f;
        grow = y >= 4.0f * hf * hf;
    } else {
        const float da = (float)c.dt_max;
        while (nd > da && nd > dmin) nd *= 0.5f;
        grow = da >= 2.0f * hf;
    }
    const long long q2 = (long long)(2.0 * h * recip_pow2(c.dt_min));
    double ndd = (double)nd;
    if (ndd == h && grow && 2.0 * h <= c.dt_max && (tnq & (q2 - 1)) == 0) ndd = 2.0 * h;
    return ndd;
}

// Records particle i's new time, next step nd and level after a step h.
__device__ __forceinline__ void commit_step(const BlockCorrect &c, int64_t i, int slot, double h, double nd,
                                            double tn, long long tnq) {
    if (c.level && nd != h) {
        atomicSub(&c.level[block_level(h, c.dt_max)], 1);
        atomicAdd(&c.level[block_level(nd, c.dt_max)], 1);
    }
    const long long tq_next = tnq + (long long)(nd * recip_pow2(c.dt_min));
    c.t[i] = tn;
    c.dt[i] = nd;
    c.tq[i] = tq_next;
    if (c.m.xr) {
        c.m.tcq[slot] = tnq;
        c.m.tq[slot] = tq_next;
    }
}

// Component d of the tile frame of j-set slot `slot` at time tnq (units of
// dt_min): its position c0 + cv (t - t0) in FP64 and its velocity cv.
__device__ __forceinline__ void frame_component(const BlockCorrect &c, int slot, int d, long long tnq, double &fc,
                                                double &fv) {
    const int tile = slot / c.m.tc;
    fv = (double)reinterpret_cast<const float *>(c.m.vchl + 2 * tile)[d];
    fc = fma(fv, (double)(tnq - c.sc->frame_t0q) * c.dt_min, c.m.c0[(int64_t)d * c.m.n_tiles + tile]);
}

// The slot's mirror after a correction to time tnq (F32C): offsets from the
// frame (fc, fv: the frame's position and velocity component at tnq).
__device__ __forceinline__ void mirror_store(const BlockCorrect &c, int slot, int d, double x1, double v1,
                                             double a1, double j1, double fc, double fv) {
    const int64_t qs = d * c.m.n_pad + slot;
    const double xr = x1 - fc;
    const float hi = (float)xr;
    c.m.xr[qs] = hi;
    c.m.xl[qs] = (float)(xr - (double)hi);
    c.m.vr[qs] = (float)(v1 - fv);
    c.m.af[qs] = (float)a1;
    c.m.jf[qs] = (float)j1;
}

// Hermite corrector of active particle (row) i over its step h = dt_i with the
// new acceleration A1, jerk J1 and potential p1, then its next step by
// Aarseth's criterion.  Steps are powers of two >= dt_min and t_next is a
// multiple of dt_min, so dividing by h, h^2, h^3 is the exact multiplication
// by their reciprocals and "t_next is a multiple of 2h" is an integer test;
// both give the oracle's results bit for bit.  F32C (the F32C path): h^2/12
// is rounded once and multiplied (within an ulp of the quotient the oracle
// takes, against the pair sums' 1e-7), and the criterion runs in FP32
// (criterion_step_f32).
template <bool F32C>
__device__ __forceinline__ void correct_particle(const BlockCorrect &c, int64_t i, int slot,
                                                 const double (&A1)[3], const double (&J1)[3], double p1,
                                                 double tn, long long tnq) {
    const double h = c.dt[i], h2 = h * h;
    const double ih = recip_pow2(h), ih2 = ih * ih, ih3 = ih2 * ih;
    const double c12 = h2 * (1.0 / 12.0);  // = RN(h^2 / 12) for a power-of-two h
    double A2[3], A3[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int64_t q = d * c.n + i;
        const double a0 = c.acc[q], j0 = c.jerk[q], v0 = c.vel[q];
        double v1, x1;
        if (F32C) {
            v1 = v0 + (a0 + A1[d]) * h / 2.0 + (j0 - J1[d]) * c12;
            x1 = c.pos[q] + (v0 + v1) * h / 2.0 + (a0 - A1[d]) * c12;
        } else {
            v1 = v0 + (a0 + A1[d]) * h / 2.0 + (j0 - J1[d]) * h2 / 12.0;
            x1 = c.pos[q] + (v0 + v1) * h / 2.0 + (a0 - A1[d]) * h2 / 12.0;
        }
        c.pos[q] = x1;
        c.vel[q] = v1;
        A3[d] = (12.0 * (a0 - A1[d]) + 6.0 * h * (j0 + J1[d])) * ih3;
        A2[d] = (-6.0 * (a0 - A1[d]) - h * (4.0 * j0 + 2.0 * J1[d])) * ih2 + h * A3[d];
        c.acc[q] = A1[d];
        c.jerk[q] = J1[d];
        if (c.m.xr) {
            double fc, fv;
            frame_component(c, slot, d, tnq, fc, fv);
            mirror_store(c, slot, d, x1, v1, A1[d], J1[d], fc, fv);
        }
    }
    if (c.pot) c.pot[i] = p1;
    const double sa = A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2];
    const double sj = J1[0] * J1[0] + J1[1] * J1[1] + J1[2] * J1[2];
    const double s2 = A2[0] * A2[0] + A2[1] * A2[1] + A2[2] * A2[2];
    const double s3 = A3[0] * A3[0] + A3[1] * A3[1] + A3[2] * A3[2];
    const double nd = F32C ? criterion_step_f32(c, h, sa, sj, s2, s3, tnq)
                           : criterion_step(c, h, sqrt(sa), sqrt(sj), sqrt(s2), sqrt(s3), tnq);
    commit_step(c, i, slot, h, nd, tn, tnq);
}

// correct_particle spread over four consecutive lanes of a warp: lane sub
// (0..2) corrects component sub, the norms are summed across the three lanes
// in component order, and lane 0 chooses the step.  Every lane of the warp
// calls it (the shuffles need them); lanes with valid == false store nothing.
// The particle's step h, its component sub of a0, j0, v0, x0 and (with a
// mirror) of its tile frame at tnq, fc and fv, come in as arguments (loaded
// ahead of time by the caller, or by correct_particle_x4).
template <bool F32C>
__device__ __forceinline__ void correct_particle_x4_pre(const BlockCorrect &c, int64_t i, int slot, bool valid,
                                                        int sub, double h, double a0, double j0, double v0,
                                                        double x0, double fc, double fv, double a1, double j1,
                                                        double p1, double tn, long long tnq) {
    const double h2 = h * h;
    const double ih = recip_pow2(h), ih2 = ih * ih, ih3 = ih2 * ih;
    double sq[4] = {0.0, 0.0, 0.0, 0.0};  // this component's a1^2, j1^2, a2^2, a3^2
    if (sub < 3) {
        const int64_t q = sub * c.n + i;
        double v1, x1;
        if (F32C) {
            const double c12 = h2 * (1.0 / 12.0);  // = RN(h^2 / 12) for a power-of-two h
            v1 = v0 + (a0 + a1) * h / 2.0 + (j0 - j1) * c12;
            x1 = x0 + (v0 + v1) * h / 2.0 + (a0 - a1) * c12;
        } else {
            v1 = v0 + (a0 + a1) * h / 2.0 + (j0 - j1) * h2 / 12.0;
            x1 = x0 + (v0 + v1) * h / 2.0 + (a0 - a1) * h2 / 12.0;
        }
        const double a3 = (12.0 * (a0 - a1) + 6.0 * h * (j0 + j1)) * ih3;
        const double a2 = (-6.0 * (a0 - a1) - h * (4.0 * j0 + 2.0 * j1)) * ih2 + h * a3;
        if (valid) {
            c.pos[q] = x1;
            c.vel[q] = v1;
            c.acc[q] = a1;
            c.jerk[q] = j1;
            if (c.m.xr) mirror_store(c, slot, sub, x1, v1, a1, j1, fc, fv);
        }
        sq[0] = a1 * a1;
        sq[1] = j1 * j1;
        sq[2] = a2 * a2;
        sq[3] = a3 * a3;
    }
    const int lane = threadIdx.x % 32, base = lane & ~3;
    double nrm[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double x = __shfl_sync(0xffffffffu, sq[k], base);
        const double y = __shfl_sync(0xffffffffu, sq[k], base + 1);
        const double z = __shfl_sync(0xffffffffu, sq[k], base + 2);
        nrm[k] = x + y + z;  // squared norm
    }
    if (sub != 0 || !valid) return;
    if (c.pot) c.pot[i] = p1;
    const double nd = F32C ? criterion_step_f32(c, h, nrm[0], nrm[1], nrm[2], nrm[3], tnq)
                           : criterion_step(c, h, sqrt(nrm[0]), sqrt(nrm[1]), sqrt(nrm[2]), sqrt(nrm[3]), tnq);
    commit_step(c, i, slot, h, nd, tn, tnq);
}

template <bool F32C>
__device__ __forceinline__ void correct_particle_x4(const BlockCorrect &c, int64_t i, int slot, bool valid,
                                                    int sub, double a1, double j1, double p1, double tn,
                                                    long long tnq) {
    const double h = c.dt[i];
    double a0 = 0.0, j0 = 0.0, v0 = 0.0, x0 = 0.0, fc = 0.0, fv = 0.0;
    if (sub < 3) {
        const int64_t q = sub * c.n + i;
        a0 = c.acc[q];
        j0 = c.jerk[q];
        v0 = c.vel[q];
        x0 = c.pos[q];
        if (c.m.xr) frame_component(c, slot, sub, tnq, fc, fv);
    }
    correct_particle_x4_pre<F32C>(c, i, slot, valid, sub, h, a0, j0, v0, x0, fc, fv, a1, j1, p1, tn, tnq);
}

// FP64 epilogue of one active particle of the F32C path: scale by G, then correct the particle
// (corr.sc set) or store a1, j1, p1 at its row.
__device__ __forceinline__ void subset_finalize(const F32CJerkParams &p, const BlockCorrect &corr,
                                                int slot, const double (&r)[7]) {
    const int64_t u = p.perm[slot];
    const double ph = r[6];
    if (corr.sc) {
        const double A1[3] = {p.G * r[0], p.G * r[1], p.G * r[2]};
        const double J1[3] = {p.G * r[3], p.G * r[4], p.G * r[5]};
        correct_particle<true>(corr, u, slot, A1, J1, -p.G * ph, corr.sc->t_next, corr.sc->t_next_q);
        return;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p.acc[d * p.n + u] = p.G * r[d];
        p.jerk[d * p.n + u] = p.G * r[3 + d];
    }
    if (p.pot) p.pot[u] = -p.G * ph;
}

}  // namespace nbody
