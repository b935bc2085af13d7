// forces_f32c.cuh -- the FP32-compensated direct-summation force kernel (sm_103a).
//
// Computes the Sec. 3 force sum (divided by m_i, Plummer-softened) for every
// packed i-slot of the work items it takes from a queue:
//
//   a_i   =  G sum_j m_j (r_j - r_i) (|r_j - r_i|^2 + eps^2)^(-3/2)
//   phi_i = -G sum_j m_j             (|r_j - r_i|^2 + eps^2)^(-1/2)
//
// Design (GB300):
//   * Persistent CTAs: each takes (cluster, i-tile, j-range) items from an
//     atomic queue head until the queue is empty.  One i-tile = the CTA's
//     block*p particles, which also share one centre.
//   * Each thread holds p i-particles in registers.  j-particles stream through
//     shared memory in tiles of tj as SoA float arrays (x, y, z, m), double
//     buffered: the next tile's global loads are issued before the current
//     tile is consumed.  All lanes read the same shared address (broadcast).
//   * Paired FP32 arithmetic: two consecutive j-particles are processed by one
//     f32x2 instruction (__fadd2_rn / __ffma2_rn / __fmul2_rn), so one issue
//     slot drives two FP32 lanes and the per-pair issue budget leaves room for
//     the MUFU rsqrt and the shared loads.  Per pair: 3 add (dx), 3 fma (r^2,
//     eps^2 folded in), 1 rsqrt, 3 mul (m s, s^2, m s^3), 1 add (phi),
//     3 fma (a) = 13 FP32 operations + 1 MUFU.
//   * Precision: coordinates are FP32 offsets from each tile's centre, which
//     is held as an unevaluated float pair hi + lo (48 significant bits).  Per
//     j-tile the centre difference c_I - c_J is formed as a float pair by an
//     error-free TwoSum (exactly 0 on the diagonal tile) and added to each i
//     offset as two rounded adds, so close pairs keep their digits whatever the
//     absolute position, the rounding of the shift is per particle (not one
//     coherent displacement of a whole tile pair), and the tile loop runs no
//     FP64 instruction.  Each thread sums a tile's terms in
//     FP32 (the potential terms of each eight j's as a tree first), then
//     folds the tile sum into a Kahan-compensated FP32 accumulator;
//     sum - compensation is converted to FP64 at the end.
//   * Split j-ranges (small N or load balance): each split writes its FP64
//     partials; the CTA that finishes last (atomic ticket, no waiting) adds
//     them in split order, so the result is bitwise deterministic.
//   * Self pair: on the diagonal j-tiles (those of the CTA's own centre tile)
//     each thread drops the potential term of its own slot before it enters
//     the FP32 tile sum (its acceleration term is exactly 0: the separation is
//     0); every other j-tile runs the unmasked loop.  With eps = 0 the r^2 > 0
//     guard already gives the self pair (and coincident pairs) zero.
//   * Epilogue in FP64: scale by G, scatter to the caller's row through perm,
//     and optionally apply the closing half-kick.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nbody_internal.h"

namespace nbody {

__device__ __forceinline__ float rsqrt_mufu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Centre difference (ih + il) - (jh + jl) as an unevaluated float pair hi + lo,
// accurate to ~2^-48 relative (Knuth's error-free TwoSum on the hi parts).  The
// shift is then applied to each i-offset as two rounded adds, so its rounding
// is per particle rather than one common displacement of the whole tile.
__device__ __forceinline__ void centre_diff(float ih, float il, float jh, float jl, float &hi,
                                            float &lo) {
    const float s = __fsub_rn(ih, jh);
    const float bb = __fsub_rn(s, ih);
    const float e = __fadd_rn(__fsub_rn(ih, __fsub_rn(s, bb)), __fsub_rn(-jh, bb));
    hi = s;
    lo = __fadd_rn(e, __fsub_rn(il, jl));
}

// Folds one tile's FP32 sum x into the running sum s with Kahan compensation c.
// NBODY_TILE_SUM_COMPENSATION=0 (an accuracy ablation: build.py builds it only
// on request, as libnbody_ablate_tile_sums.so) folds with a plain FP32 add.
#ifndef NBODY_TILE_SUM_COMPENSATION
#define NBODY_TILE_SUM_COMPENSATION 1
#endif
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
#if NBODY_TILE_SUM_COMPENSATION
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
#else
    c = 0.0f;
    s = __fadd_rn(s, x);
#endif
}

// TREE: potential terms added as a tree before they join the running sum, 4
// (eight j's) or 2 (four j's) at a time; 4 needs 8 more registers per
// i-particle held at once.
template <int BLOCK, int P, int TJ, bool EPS_ZERO, int TREE = 4>
struct F32CKernel {
    static_assert(TREE == 2 || TREE == 4, "tree of two or four potential terms");
    static constexpr int TC = BLOCK * P;
    static constexpr int NV = TJ;  // float4 vectors per j-tile (4 arrays x TJ/4)
    static constexpr int NLD = (NV + BLOCK - 1) / BLOCK;
    static_assert(TJ % 8 == 0, "tj must be a multiple of 8");
    static_assert(TC % TJ == 0, "a j-tile must not straddle two centre tiles");

    struct Smem {
        float4 j[2][4][TJ / 4];  // [buffer][x|y|z|m][TJ/4]
        float shift[2][8];       // hi (0..2) and lo (4..6) of the centre difference
        int item;
        int last;
    };

    __device__ static __forceinline__ void load_tile(const F32CParams &p, int gs, float4 (&r)[NLD]) {
#pragma unroll
        for (int q = 0; q < NLD; ++q) {
            const int v = threadIdx.x + q * BLOCK;
            if (NV % BLOCK == 0 || v < NV) {
                const int arr = v / (TJ / 4);
                const int off = (v % (TJ / 4)) * 4;
                const float *base = arr == 0 ? p.px : arr == 1 ? p.py : arr == 2 ? p.pz : p.pm;
                r[q] = __ldg(reinterpret_cast<const float4 *>(base + gs + off));
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

    // Offset that moves i-tile coordinates into the j-tile's frame, c_I - c_J,
    // as a float pair (see centre_diff).
    __device__ static __forceinline__ void store_shift(Smem &sm, int b, float4 ih, float4 il,
                                                       float4 jh, float4 jl) {
        centre_diff(ih.x, il.x, jh.x, jl.x, sm.shift[b][0], sm.shift[b][4]);
        centre_diff(ih.y, il.y, jh.y, jl.y, sm.shift[b][1], sm.shift[b][5]);
        centre_diff(ih.z, il.z, jh.z, jl.z, sm.shift[b][2], sm.shift[b][6]);
    }

    // One pair of j's (the halves of each float2, tile positions j0 and j0 + 1)
    // against the thread's P i-particles: accumulates the acceleration terms
    // and returns the potential terms m_j s in mo (summed by the caller).
    // MASK: d[k] is the tile position of i-particle k's own slot (or outside
    // the tile), whose potential term is dropped.
    template <bool MASK>
    __device__ static __forceinline__ void body(float2 xj, float2 yj, float2 zj, float2 mj,
                                                const float2 e2, const float2 (&nx)[P],
                                                const float2 (&ny)[P], const float2 (&nz)[P],
                                                float2 (&ax)[P], float2 (&ay)[P], float2 (&az)[P],
                                                float2 (&mo)[P], const int (&d)[P], int j0) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const float2 dx = __fadd2_rn(xj, nx[k]);
            const float2 dy = __fadd2_rn(yj, ny[k]);
            const float2 dz = __fadd2_rn(zj, nz[k]);
            float2 r2 = __ffma2_rn(dx, dx, e2);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            float2 s;
            if (EPS_ZERO) {
                s.x = r2.x > 0.0f ? rsqrt_mufu(r2.x) : 0.0f;
                s.y = r2.y > 0.0f ? rsqrt_mufu(r2.y) : 0.0f;
            } else {
                s.x = rsqrt_mufu(r2.x);
                s.y = rsqrt_mufu(r2.y);
            }
            const float2 ms = __fmul2_rn(mj, s);
            const float2 s2 = __fmul2_rn(s, s);
            const float2 w3 = __fmul2_rn(ms, s2);
            float2 mp = ms;
            if (MASK) {
                mp.x = d[k] == j0 ? 0.0f : ms.x;
                mp.y = d[k] == j0 + 1 ? 0.0f : ms.y;
            }
            mo[k] = mp;
            ax[k] = __ffma2_rn(w3, dx, ax[k]);
            ay[k] = __ffma2_rn(w3, dy, ay[k]);
            az[k] = __ffma2_rn(w3, dz, az[k]);
        }
    }

    // All pairs of one shared-memory j-tile (buffer b) against the thread's P
    // i-particles, summed in FP32.  2 * TREE j's per iteration; their TREE
    // potential terms per lane are added as a tree before they join the
    // running sum (the same number of adds: a shorter loop-carried chain and
    // smaller rounding errors).
    template <bool MASK>
    __device__ static __forceinline__ void tile_pass(const Smem &sm, int b, const float2 e2,
                                                     const float2 (&nx)[P], const float2 (&ny)[P],
                                                     const float2 (&nz)[P], float2 (&ax)[P],
                                                     float2 (&ay)[P], float2 (&az)[P],
                                                     float2 (&ph)[P], const int (&d)[P]) {
        static_assert((TJ / 4) % 2 == 0, "two float4 columns per iteration");
        const float4 *jx = sm.j[b][0];
        const float4 *jy = sm.j[b][1];
        const float4 *jz = sm.j[b][2];
        const float4 *jm = sm.j[b][3];
        if (TREE == 2) {
#pragma unroll 2
            for (int v = 0; v < TJ / 4; ++v) {
                float2 m0[P], m1[P];
                const float4 X = jx[v], Y = jy[v], Z = jz[v], M = jm[v];
                body<MASK>(make_float2(X.x, X.y), make_float2(Y.x, Y.y), make_float2(Z.x, Z.y),
                           make_float2(M.x, M.y), e2, nx, ny, nz, ax, ay, az, m0, d, 4 * v);
                body<MASK>(make_float2(X.z, X.w), make_float2(Y.z, Y.w), make_float2(Z.z, Z.w),
                           make_float2(M.z, M.w), e2, nx, ny, nz, ax, ay, az, m1, d, 4 * v + 2);
#pragma unroll
                for (int k = 0; k < P; ++k) ph[k] = __fadd2_rn(ph[k], __fadd2_rn(m0[k], m1[k]));
            }
            return;
        }
        // two iterations in flight on the 1024-wide tiles (measured 0.8 % faster
        // there, not on narrower ones)
        constexpr int kUnroll = TJ >= 1024 ? 2 : 1;
#pragma unroll kUnroll
        for (int v = 0; v < TJ / 4; v += 2) {
            float2 m0[P], m1[P], m2[P], m3[P];
            {
                const float4 X = jx[v], Y = jy[v], Z = jz[v], M = jm[v];
                body<MASK>(make_float2(X.x, X.y), make_float2(Y.x, Y.y), make_float2(Z.x, Z.y),
                           make_float2(M.x, M.y), e2, nx, ny, nz, ax, ay, az, m0, d, 4 * v);
                body<MASK>(make_float2(X.z, X.w), make_float2(Y.z, Y.w), make_float2(Z.z, Z.w),
                           make_float2(M.z, M.w), e2, nx, ny, nz, ax, ay, az, m1, d, 4 * v + 2);
            }
            {
                const float4 X = jx[v + 1], Y = jy[v + 1], Z = jz[v + 1], M = jm[v + 1];
                body<MASK>(make_float2(X.x, X.y), make_float2(Y.x, Y.y), make_float2(Z.x, Z.y),
                           make_float2(M.x, M.y), e2, nx, ny, nz, ax, ay, az, m2, d, 4 * v + 4);
                body<MASK>(make_float2(X.z, X.w), make_float2(Y.z, Y.w), make_float2(Z.z, Z.w),
                           make_float2(M.z, M.w), e2, nx, ny, nz, ax, ay, az, m3, d, 4 * v + 6);
            }
#pragma unroll
            for (int k = 0; k < P; ++k)
                ph[k] = __fadd2_rn(ph[k], __fadd2_rn(__fadd2_rn(m0[k], m1[k]), __fadd2_rn(m2[k], m3[k])));
        }
    }

    // FP64 epilogue for one i-slot: scale, scatter, kick.
    __device__ static __forceinline__ void finalize(const F32CParams &p, const ClusterDev &cl,
                                                    int slot, double sx, double sy, double sz,
                                                    double sp) {
        const int local = slot - cl.slot_begin;
        if (local >= cl.n) return;
        const int64_t u = p.perm[slot];
        const double a0 = p.G * sx, a1 = p.G * sy, a2 = p.G * sz;
        p.acc[u] = a0;
        p.acc[p.n + u] = a1;
        p.acc[2 * p.n + u] = a2;
        if (p.pot) p.pot[u] = -p.G * sp;
        if (p.vel) {
            p.vel[u] += p.half_dt * a0;
            p.vel[p.n + u] += p.half_dt * a1;
            p.vel[2 * p.n + u] += p.half_dt * a2;
        }
    }

    __device__ static void run(const F32CParams p) {
        __shared__ Smem sm;
        const float2 zero2 = make_float2(0.0f, 0.0f);
        for (;;) {
            if (threadIdx.x == 0) sm.item = atomicAdd(p.counters, 1);
            __syncthreads();
            const int item_idx = sm.item;
            if (item_idx >= p.n_items) break;
            const Item it = p.items[item_idx];
            const ClusterDev cl = p.cl[it.cluster];
            const int ibase = it.tile * TC;
            const float2 e2 = make_float2(cl.eps2f, cl.eps2f);
            const float4 cih = p.chl[2 * it.tile + 0];  // centre of the i-tile, hi part
            const float4 cil = p.chl[2 * it.tile + 1];  // lo part

            float ox[P], oy[P], oz[P];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int slot = ibase + threadIdx.x + k * BLOCK;
                ox[k] = p.px[slot];
                oy[k] = p.py[slot];
                oz[k] = p.pz[slot];
            }
            float ksum[P][4], kcmp[P][4];
#pragma unroll
            for (int k = 0; k < P; ++k)
#pragma unroll
                for (int c = 0; c < 4; ++c) ksum[k][c] = kcmp[k][c] = 0.0f;

            const int ntj = it.jt1 - it.jt0;
            float4 reg[NLD];
            float4 cjh = make_float4(0.f, 0.f, 0.f, 0.f), cjl = cjh;
            {
                const int gs = cl.slot_begin + it.jt0 * TJ;
                load_tile(p, gs, reg);
                store_tile(sm, 0, reg);
                if (threadIdx.x == 0) {
                    const int jc = gs / TC;
                    store_shift(sm, 0, cih, cil, p.chl[2 * jc], p.chl[2 * jc + 1]);
                }
            }
            __syncthreads();

            for (int t = 0; t < ntj; ++t) {
                const int b = t & 1;
                const bool more = t + 1 < ntj;
                const int gsn = cl.slot_begin + (it.jt0 + t + 1) * TJ;
                if (more) load_tile(p, gsn, reg);
                if (more && threadIdx.x == 0) {
                    const int jc = gsn / TC;  // loads issued now, used after the tile
                    cjh = p.chl[2 * jc];
                    cjl = p.chl[2 * jc + 1];
                }
                float2 nx[P], ny[P], nz[P];
                {
                    const float sx = sm.shift[b][0], sy = sm.shift[b][1], sz = sm.shift[b][2];
                    const float lx = sm.shift[b][4], ly = sm.shift[b][5], lz = sm.shift[b][6];
#pragma unroll
                    for (int k = 0; k < P; ++k) {
                        const float qx = -__fadd_rn(__fadd_rn(ox[k], sx), lx);
                        const float qy = -__fadd_rn(__fadd_rn(oy[k], sy), ly);
                        const float qz = -__fadd_rn(__fadd_rn(oz[k], sz), lz);
                        nx[k] = make_float2(qx, qx);
                        ny[k] = make_float2(qy, qy);
                        nz[k] = make_float2(qz, qz);
                    }
                }
                float2 ax[P], ay[P], az[P], ph[P];
#pragma unroll
                for (int k = 0; k < P; ++k) ax[k] = ay[k] = az[k] = ph[k] = zero2;

                // diagonal j-tile (inside the CTA's own centre tile): mask the
                // self pair's potential term (CTA-uniform branch)
                const int gs = cl.slot_begin + (it.jt0 + t) * TJ;
                int d[P];
#pragma unroll
                for (int k = 0; k < P; ++k) d[k] = ibase + threadIdx.x + k * BLOCK - gs;
                if (!EPS_ZERO && gs / TC == it.tile)
                    tile_pass<true>(sm, b, e2, nx, ny, nz, ax, ay, az, ph, d);
                else
                    tile_pass<false>(sm, b, e2, nx, ny, nz, ax, ay, az, ph, d);
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    kahan_add(ksum[k][0], kcmp[k][0], __fadd_rn(ax[k].x, ax[k].y));
                    kahan_add(ksum[k][1], kcmp[k][1], __fadd_rn(ay[k].x, ay[k].y));
                    kahan_add(ksum[k][2], kcmp[k][2], __fadd_rn(az[k].x, az[k].y));
                    kahan_add(ksum[k][3], kcmp[k][3], __fadd_rn(ph[k].x, ph[k].y));
                }
                if (more) {
                    store_tile(sm, b ^ 1, reg);
                    if (threadIdx.x == 0) store_shift(sm, b ^ 1, cih, cil, cjh, cjl);
                }
                __syncthreads();
            }

            // compensated FP32 sums -> FP64 (sum - compensation is exact in FP64)
            double res[P][4];
#pragma unroll
            for (int k = 0; k < P; ++k)
#pragma unroll
                for (int c = 0; c < 4; ++c) res[k][c] = (double)ksum[k][c] - (double)kcmp[k][c];

            if (it.nsplit <= 1) {
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const int slot = ibase + threadIdx.x + k * BLOCK;
                    finalize(p, cl, slot, res[k][0], res[k][1], res[k][2], res[k][3]);
                }
                continue;  // the loop head's __syncthreads orders sm.item reuse
            }

            double *mine = p.partial + (size_t)(it.pbase + it.split) * 4 * TC;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int l = threadIdx.x + k * BLOCK;
#pragma unroll
                for (int c = 0; c < 4; ++c) __stcg(mine + c * TC + l, res[k][c]);
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
                double acc4[4] = {0.0, 0.0, 0.0, 0.0};
                for (int s = 0; s < it.nsplit; ++s) {
                    const double *ps = p.partial + (size_t)(it.pbase + s) * 4 * TC;
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc4[c] += __ldcg(ps + c * TC + l);
                }
                const int slot = ibase + l;
                finalize(p, cl, slot, acc4[0], acc4[1], acc4[2], acc4[3]);
            }
        }
    }
};

// The tree of four where the register budget allows it: one CTA per SM (255
// registers) or two i-particles per thread; two otherwise.
template <int BLOCK, int P, int TJ, int MINB, bool EPS_ZERO>
__global__ void __launch_bounds__(BLOCK, MINB) forces_f32c_kernel(const F32CParams p) {
    F32CKernel<BLOCK, P, TJ, EPS_ZERO, (P <= 2 || MINB <= 2) ? 4 : 2>::run(p);
}

}  // namespace nbody
