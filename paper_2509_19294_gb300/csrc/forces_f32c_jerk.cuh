// forces_f32c_jerk.cuh -- FP32-compensated acceleration + jerk kernel (sm_103a).
//
// The paper's device kernel computes the acceleration together with its first
// time derivative, the jerk (Sec. 3).  With r = r_j - r_i, u = v_j - v_i,
// s = (|r|^2 + eps^2)^(-1/2):
//
//   a_i    =  G sum_j m_j s^3 r
//   jerk_i =  G sum_j m_j s^3 (u - 3 (r . u) s^2 r)
//   phi_i  = -G sum_j m_j s
//
// Same design as the acceleration kernel (forces_f32c.cuh): persistent CTAs over
// the (cluster, i-tile, j-range) queue, p i-particles per thread, j-tiles in
// double-buffered shared memory, two j-particles per f32x2 instruction, FP32
// offsets from float-pair tile centres for positions AND velocities, Kahan-
// compensated per-tile sums, FP64 split reduction and epilogue; centre
// differences as float pairs added per particle, the self pair's potential term
// masked on the diagonal j-tiles (see forces_f32c.cuh).  Per pair:
// 3 add (r), 3 add (u), 3 fma (r^2), 3 (r.u), 1 rsqrt, 3 mul (m s, s^2, m s^3),
// 2 mul (beta = -3 (r.u) s^2), 1 add (phi), 3 fma (a), 6 fma (jerk) =
// 27 FP32 operations + 1 MUFU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "forces_f32c.cuh"
#include "nbody_internal.h"

namespace nbody {

template <int BLOCK, int P, int TJ, bool EPS_ZERO>
struct F32CJerkKernel {
    static constexpr int TC = BLOCK * P;
    static constexpr int NA = 7;                 // x, y, z, m, vx, vy, vz
    static constexpr int NV = NA * TJ / 4;       // float4 vectors per j-tile
    static constexpr int NLD = (NV + BLOCK - 1) / BLOCK;
    static constexpr int NC = 7;                 // ax, ay, az, jx, jy, jz, phi
    static_assert(TJ % 8 == 0, "tj must be a multiple of 8");

    struct Smem {
        float4 j[2][NA][TJ / 4];
        float shift[2][12];  // hi, lo of the position shift (0..2, 3..5) and velocity shift (6..8, 9..11)
        int item;
        int last;
    };

    __device__ static __forceinline__ const float *array(const F32CJerkParams &p, int a) {
        return a == 0 ? p.px : a == 1 ? p.py : a == 2 ? p.pz : a == 3 ? p.pm
             : a == 4 ? p.pvx : a == 5 ? p.pvy : p.pvz;
    }

    __device__ static __forceinline__ void load_tile(const F32CJerkParams &p, int gs, float4 (&r)[NLD]) {
#pragma unroll
        for (int q = 0; q < NLD; ++q) {
            const int v = threadIdx.x + q * BLOCK;
            if (NV % BLOCK == 0 || v < NV) {
                const int a = v / (TJ / 4);
                const int off = (v % (TJ / 4)) * 4;
                r[q] = __ldg(reinterpret_cast<const float4 *>(array(p, a) + gs + off));
            }
        }
    }

    __device__ static __forceinline__ void store_tile(Smem &sm, int b, const float4 (&r)[NLD]) {
#pragma unroll
        for (int q = 0; q < NLD; ++q) {
            const int v = threadIdx.x + q * BLOCK;
            if (NV % BLOCK == 0 || v < NV) sm.j[b][v / (TJ / 4)][v % (TJ / 4)] = r[q];
        }
    }

    __device__ static __forceinline__ void store_shift(Smem &sm, int b, const float4 (&ic)[4],
                                                       const float4 (&jc)[4]) {
        // ic/jc: position hi, position lo, velocity hi, velocity lo
        float *sh = sm.shift[b];
        centre_diff(ic[0].x, ic[1].x, jc[0].x, jc[1].x, sh[0], sh[3]);
        centre_diff(ic[0].y, ic[1].y, jc[0].y, jc[1].y, sh[1], sh[4]);
        centre_diff(ic[0].z, ic[1].z, jc[0].z, jc[1].z, sh[2], sh[5]);
        centre_diff(ic[2].x, ic[3].x, jc[2].x, jc[3].x, sh[6], sh[9]);
        centre_diff(ic[2].y, ic[3].y, jc[2].y, jc[3].y, sh[7], sh[10]);
        centre_diff(ic[2].z, ic[3].z, jc[2].z, jc[3].z, sh[8], sh[11]);
    }

    __device__ static __forceinline__ void load_centres(const F32CJerkParams &p, int tile,
                                                        float4 (&c)[4]) {
        c[0] = p.chl[2 * tile];
        c[1] = p.chl[2 * tile + 1];
        c[2] = p.vchl[2 * tile];
        c[3] = p.vchl[2 * tile + 1];
    }

    // One j-pair (two consecutive j's in the halves of each float2, at tile
    // positions j0 and j0 + 1) against P i's.  MASK: d[k] is the tile position
    // of i-particle k's own slot (or outside the tile), whose potential term is
    // dropped; its acceleration and jerk terms are exactly 0 (r = u = 0).
    template <bool MASK>
    __device__ static __forceinline__ void body(const float2 (&J)[NA], const float2 e2,
                                                const float2 (&ni)[P][6], float2 (&acc)[P][NC],
                                                const int (&d)[P], int j0) {
        const float2 m3 = make_float2(-3.0f, -3.0f);
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const float2 dx = __fadd2_rn(J[0], ni[k][0]);
            const float2 dy = __fadd2_rn(J[1], ni[k][1]);
            const float2 dz = __fadd2_rn(J[2], ni[k][2]);
            const float2 ux = __fadd2_rn(J[4], ni[k][3]);
            const float2 uy = __fadd2_rn(J[5], ni[k][4]);
            const float2 uz = __fadd2_rn(J[6], ni[k][5]);
            float2 r2 = __ffma2_rn(dx, dx, e2);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            float2 rv = __fmul2_rn(dx, ux);
            rv = __ffma2_rn(dy, uy, rv);
            rv = __ffma2_rn(dz, uz, rv);
            float2 s;
            if (EPS_ZERO) {
                s.x = r2.x > 0.0f ? rsqrt_mufu(r2.x) : 0.0f;
                s.y = r2.y > 0.0f ? rsqrt_mufu(r2.y) : 0.0f;
            } else {
                s.x = rsqrt_mufu(r2.x);
                s.y = rsqrt_mufu(r2.y);
            }
            const float2 ms = __fmul2_rn(J[3], s);
            const float2 s2 = __fmul2_rn(s, s);
            const float2 w3 = __fmul2_rn(ms, s2);
            const float2 beta = __fmul2_rn(rv, __fmul2_rn(s2, m3));  // -3 (r.u) s^2
            float2 mp = ms;
            if (MASK) {
                mp.x = d[k] == j0 ? 0.0f : ms.x;
                mp.y = d[k] == j0 + 1 ? 0.0f : ms.y;
            }
            acc[k][6] = __fadd2_rn(acc[k][6], mp);
            acc[k][0] = __ffma2_rn(w3, dx, acc[k][0]);
            acc[k][1] = __ffma2_rn(w3, dy, acc[k][1]);
            acc[k][2] = __ffma2_rn(w3, dz, acc[k][2]);
            acc[k][3] = __ffma2_rn(w3, __ffma2_rn(beta, dx, ux), acc[k][3]);
            acc[k][4] = __ffma2_rn(w3, __ffma2_rn(beta, dy, uy), acc[k][4]);
            acc[k][5] = __ffma2_rn(w3, __ffma2_rn(beta, dz, uz), acc[k][5]);
        }
    }

    // All pairs of columns [v0, v1) of the shared-memory j-tile in buffer b
    // (four j's per column) against the thread's P i-particles, in FP32.
    template <bool MASK, class SM>
    __device__ static __forceinline__ void tile_pass(const SM &sm, int b, int v0, int v1,
                                                     const float2 e2, const float2 (&ni)[P][6],
                                                     float2 (&acc)[P][NC], const int (&d)[P]) {
#pragma unroll 1
        for (int v = v0; v < v1; ++v) {
            float4 Q[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) Q[a] = sm.j[b][a][v];
            float2 J[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) J[a] = make_float2(Q[a].x, Q[a].y);
            body<MASK>(J, e2, ni, acc, d, 4 * v);
#pragma unroll
            for (int a = 0; a < NA; ++a) J[a] = make_float2(Q[a].z, Q[a].w);
            body<MASK>(J, e2, ni, acc, d, 4 * v + 2);
        }
    }

    __device__ static __forceinline__ void finalize(const F32CJerkParams &p, const ClusterDev &cl,
                                                    int slot, const double (&r)[NC]) {
        const int local = slot - cl.slot_begin;
        if (local >= cl.n) return;
        const int64_t u = p.perm[slot];
        const double ph = r[6];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p.acc[d * p.n + u] = p.G * r[d];
            p.jerk[d * p.n + u] = p.G * r[3 + d];
        }
        if (p.pot) p.pot[u] = -p.G * ph;
    }

    __device__ static void run(const F32CJerkParams p) {
        static_assert(TC % TJ == 0, "a j-tile must not straddle two centre tiles");
        __shared__ Smem sm;
        for (;;) {
            if (threadIdx.x == 0) sm.item = atomicAdd(p.counters, 1);
            __syncthreads();
            const int item_idx = sm.item;
            if (item_idx >= p.n_items) break;
            const Item it = p.items[item_idx];
            const ClusterDev cl = p.cl[it.cluster];
            const int ibase = it.tile * TC;
            const float2 e2 = make_float2(cl.eps2f, cl.eps2f);
            float4 ic[4];
            load_centres(p, it.tile, ic);

            float own[P][6];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int slot = ibase + threadIdx.x + k * BLOCK;
                own[k][0] = p.px[slot];
                own[k][1] = p.py[slot];
                own[k][2] = p.pz[slot];
                own[k][3] = p.pvx[slot];
                own[k][4] = p.pvy[slot];
                own[k][5] = p.pvz[slot];
            }
            float ksum[P][NC], kcmp[P][NC];
#pragma unroll
            for (int k = 0; k < P; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) ksum[k][c] = kcmp[k][c] = 0.0f;

            const int ntj = it.jt1 - it.jt0;
            float4 reg[NLD];
            float4 jc[4];
            {
                const int gs = cl.slot_begin + it.jt0 * TJ;
                load_tile(p, gs, reg);
                store_tile(sm, 0, reg);
                if (threadIdx.x == 0) {
                    load_centres(p, gs / TC, jc);
                    store_shift(sm, 0, ic, jc);
                }
            }
            __syncthreads();

            for (int t = 0; t < ntj; ++t) {
                const int b = t & 1;
                const bool more = t + 1 < ntj;
                const int gsn = cl.slot_begin + (it.jt0 + t + 1) * TJ;
                if (more) load_tile(p, gsn, reg);
                if (more && threadIdx.x == 0) load_centres(p, gsn / TC, jc);
                float2 ni[P][6];
#pragma unroll
                for (int k = 0; k < P; ++k)
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const int h = q < 3 ? q : q + 3;  // hi at h, lo at h + 3
                        const float v =
                            -__fadd_rn(__fadd_rn(own[k][q], sm.shift[b][h]), sm.shift[b][h + 3]);
                        ni[k][q] = make_float2(v, v);
                    }
                float2 acc[P][NC];
#pragma unroll
                for (int k = 0; k < P; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc[k][c] = make_float2(0.0f, 0.0f);
                // diagonal j-tile (inside the CTA's own centre tile): mask the
                // self pair's potential term (CTA-uniform branch)
                const int gs = cl.slot_begin + (it.jt0 + t) * TJ;
                int d[P];
#pragma unroll
                for (int k = 0; k < P; ++k) d[k] = ibase + threadIdx.x + k * BLOCK - gs;
                if (!EPS_ZERO && gs / TC == it.tile)
                    tile_pass<true>(sm, b, 0, TJ / 4, e2, ni, acc, d);
                else
                    tile_pass<false>(sm, b, 0, TJ / 4, e2, ni, acc, d);
#pragma unroll
                for (int k = 0; k < P; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        kahan_add(ksum[k][c], kcmp[k][c], __fadd_rn(acc[k][c].x, acc[k][c].y));
                if (more) {
                    store_tile(sm, b ^ 1, reg);
                    if (threadIdx.x == 0) store_shift(sm, b ^ 1, ic, jc);
                }
                __syncthreads();
            }

            double res[P][NC];
#pragma unroll
            for (int k = 0; k < P; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) res[k][c] = (double)ksum[k][c] - (double)kcmp[k][c];

            if (it.nsplit <= 1) {
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const int slot = ibase + threadIdx.x + k * BLOCK;
                    finalize(p, cl, slot, res[k]);
                }
                continue;
            }
            double *mine = p.partial + (size_t)(it.pbase + it.split) * NC * TC;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int l = threadIdx.x + k * BLOCK;
#pragma unroll
                for (int c = 0; c < NC; ++c) __stcg(mine + c * TC + l, res[k][c]);
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                const int prev = atomicAdd(p.counters + 1 + it.tile, 1);
                sm.last = (prev == it.nsplit - 1);
            }
            __syncthreads();
            if (!sm.last) continue;
            __threadfence();
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int l = threadIdx.x + k * BLOCK;
                double tot[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) tot[c] = 0.0;
                for (int s = 0; s < it.nsplit; ++s) {
                    const double *ps = p.partial + (size_t)(it.pbase + s) * NC * TC;
#pragma unroll
                    for (int c = 0; c < NC; ++c) tot[c] += __ldcg(ps + c * TC + l);
                }
                const int slot = ibase + l;
                finalize(p, cl, slot, tot);
            }
        }
    }
};

template <int BLOCK, int P, int TJ, int MINB, bool EPS_ZERO>
__global__ void __launch_bounds__(BLOCK, MINB) forces_f32c_jerk_kernel(const F32CJerkParams p) {
    F32CJerkKernel<BLOCK, P, TJ, EPS_ZERO>::run(p);
}

}  // namespace nbody
