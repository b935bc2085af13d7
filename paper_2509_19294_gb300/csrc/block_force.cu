// block_force.cu -- individual (block) time steps: the force pass on the
// active subset (see block_sched.cu for the step's pipeline).  The subset
// kernels evaluate i-chunks of the active list against all j of their
// cluster, each CTA an even range of (i-chunk, j-tile) units; the tail kernel
// runs either the few-particle pass or the ordered sum of the partials of the
// i-chunks that several CTAs' ranges share.  An active particle is evaluated with
// its own j-set offset and its own tile centre: per j-tile each thread forms
// the exact centre difference for each of its particles, so the self pair's
// separation is exactly zero, as in the full kernels, and its potential term is
// masked before it enters the FP32 sums.  The corrector runs in the epilogue.
#include <algorithm>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "block_common.cuh"
#include "block_reduce.cuh"
#include "forces_f32c_jerk.cuh"
#include "nbody_internal.h"

namespace nbody {

// Asynchronous global -> shared copies (no register staging); the caller
// commits them and waits before reading the shared copy.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

namespace {

// Subset kernel: CTA w takes the w-th of the plan's even ranges of (i-chunk of
// the active list, j-tile) units, in unit order: the tail of one i-chunk's
// j-tiles, whole i-chunks, the head of another.  A CTA holds BLOCK * P active
// particles (P per thread) in G thread groups of BLOCK; all groups hold the
// same particles and each takes one G-th of every shared-memory j-tile, so a
// small active set still keeps G times more warps busy.  The groups' Kahan
// sums are added in group order (FP64, shared memory); an i-chunk covered
// whole is finalised at once, a part of one is written as an FP64 partial
// (slot 2w for the range's first i-chunk, 2w + 1 for its last) that
// subset_tail_kernel adds in CTA order.
template <int BLOCK, int P, int TJ, int G, bool EPS_ZERO>
struct SubsetKernel {
    using JK = F32CJerkKernel<BLOCK, P, TJ, EPS_ZERO>;
    static constexpr int NT = BLOCK * G;       // threads per CTA
    static constexpr int CS = BLOCK * P;       // active particles per chunk
    static constexpr int NA = JK::NA;
    static constexpr int NC = JK::NC;
    static constexpr int NV = JK::NV;
    static constexpr int NLD = (NV + NT - 1) / NT;
    static constexpr int COLS = TJ / 4 / G;    // float4 columns of a j-tile per group
    static_assert((TJ / 4) % G == 0, "a group takes whole float4 columns");

    struct Smem {
        float4 j[2][NA][TJ / 4];
        float4 jc[2][4];  // j-tile centre: position hi, lo, velocity hi, lo
        double red[G > 1 ? G : 1][NC][CS];
        int item;
    };

    __device__ static __forceinline__ void load_tile(const F32CJerkParams &p, int gs, float4 (&r)[NLD]) {
#pragma unroll
        for (int q = 0; q < NLD; ++q) {
            const int v = threadIdx.x + q * NT;
            if (NV % NT == 0 || v < NV) {
                const int a = v / (TJ / 4);
                const int off = (v % (TJ / 4)) * 4;
                r[q] = __ldg(reinterpret_cast<const float4 *>(JK::array(p, a) + gs + off));
            }
        }
    }

    __device__ static __forceinline__ void store_tile(Smem &sm, int b, const float4 (&r)[NLD]) {
#pragma unroll
        for (int q = 0; q < NLD; ++q) {
            const int v = threadIdx.x + q * NT;
            if (NV % NT == 0 || v < NV) sm.j[b][v / (TJ / 4)][v % (TJ / 4)] = r[q];
        }
    }

    __device__ static void run(const F32CSubsetParams q) {
        __shared__ Smem sm;
        const F32CJerkParams &p = q.base;
        // CTA w takes the w-th of nw even ranges of the W units
        const int nw = *q.n_items;
        if ((int)blockIdx.x >= nw) return;
        const long long W = q.sc->n_units;
        const int w = blockIdx.x;
        const long long u0 = even_range_begin(w, W, nw), u1 = even_range_begin(w + 1, W, nw);
        const int li = threadIdx.x % BLOCK, g = threadIdx.x / BLOCK;
        for (long long u = u0, unext = u0; u < u1; u = unext) {
            SubItem it;
            {
                int lo = 0, hi = q.ncl;  // cluster: the last c with work_off[c] <= u
                while (hi - lo > 1) {
                    const int mid = (lo + hi) / 2;
                    if (q.work_off[mid] <= u) lo = mid;
                    else hi = mid;
                }
                const int n_jt = p.cl[lo].n_jt;
                const long long local = u - q.work_off[lo];
                const int ci = (int)(local / n_jt), t = (int)(local % n_jt);
                const int t1 = (int)min((long long)n_jt, t + (u1 - u));
                it.cluster = lo;
                it.a0 = q.act_begin[lo] + ci * CS;
                it.na = min(CS, q.act_n[lo] - ci * CS);
                it.chunk = q.ich_off[lo] + ci;
                it.jt0 = t;
                it.jt1 = t1;
                it.nsplit = (t == 0 && t1 == n_jt) ? 1 : 2;  // 1: the whole j range
                it.pbase = (int)even_range_slot(w, u - t, W, nw);  // the partial's slot
                it.split = 0;
                unext = u + (t1 - t);
            }
            const ClusterDev cl = p.cl[it.cluster];
            const float2 e2 = make_float2(cl.eps2f, cl.eps2f);
            int slot[P];
            bool valid[P];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int pos = li + k * BLOCK;
                valid[k] = pos < it.na;
                slot[k] = q.act_slot[it.a0 + (valid[k] ? pos : 0)];
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
                    JK::load_centres(p, gs / q.tcj, jc);
#pragma unroll
                    for (int a = 0; a < 4; ++a) sm.jc[0][a] = jc[a];
                }
            }
            __syncthreads();
            for (int t = 0; t < ntj; ++t) {
                const int b = t & 1;
                const bool more = t + 1 < ntj;
                const int gsn = cl.slot_begin + (it.jt0 + t + 1) * TJ;
                if (more) load_tile(p, gsn, reg);
                if (more && threadIdx.x == 0) JK::load_centres(p, gsn / q.tcj, jc);
                float2 ni[P][6];
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    float4 ic[4];
                    JK::load_centres(p, slot[k] / q.tcj, ic);
                    const float own[6] = {p.px[slot[k]], p.py[slot[k]], p.pz[slot[k]],
                                          p.pvx[slot[k]], p.pvy[slot[k]], p.pvz[slot[k]]};
                    const float ih[6] = {ic[0].x, ic[0].y, ic[0].z, ic[2].x, ic[2].y, ic[2].z};
                    const float il[6] = {ic[1].x, ic[1].y, ic[1].z, ic[3].x, ic[3].y, ic[3].z};
                    const float jh[6] = {sm.jc[b][0].x, sm.jc[b][0].y, sm.jc[b][0].z,
                                         sm.jc[b][2].x, sm.jc[b][2].y, sm.jc[b][2].z};
                    const float jl[6] = {sm.jc[b][1].x, sm.jc[b][1].y, sm.jc[b][1].z,
                                         sm.jc[b][3].x, sm.jc[b][3].y, sm.jc[b][3].z};
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        float hi, lo;
                        centre_diff(ih[c], il[c], jh[c], jl[c], hi, lo);
                        const float v = -__fadd_rn(__fadd_rn(own[c], hi), lo);
                        ni[k][c] = make_float2(v, v);
                    }
                }
                float2 acc[P][NC];
#pragma unroll
                for (int k = 0; k < P; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc[k][c] = make_float2(0.0f, 0.0f);
                // a j-tile holding one of the warp's own slots masks the self
                // pairs' potential terms (warp-uniform branch; the active
                // list is in slot order, so few tiles take it)
                const int gs = cl.slot_begin + (it.jt0 + t) * TJ;
                int d[P];
                bool own_here = false;
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    d[k] = slot[k] - gs;
                    own_here |= d[k] >= 0 && d[k] < TJ;
                }
                if (!EPS_ZERO && __any_sync(0xffffffffu, own_here))
                    JK::template tile_pass<true>(sm, b, g * COLS, (g + 1) * COLS, e2, ni, acc, d);
                else
                    JK::template tile_pass<false>(sm, b, g * COLS, (g + 1) * COLS, e2, ni, acc, d);
#pragma unroll
                for (int k = 0; k < P; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        kahan_add(ksum[k][c], kcmp[k][c], __fadd_rn(acc[k][c].x, acc[k][c].y));
                if (more) {
                    store_tile(sm, b ^ 1, reg);
                    if (threadIdx.x == 0)
#pragma unroll
                        for (int a = 0; a < 4; ++a) sm.jc[b ^ 1][a] = jc[a];
                }
                __syncthreads();
            }
            double res[P][NC];
#pragma unroll
            for (int k = 0; k < P; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) res[k][c] = (double)ksum[k][c] - (double)kcmp[k][c];
            if (G > 1) {
#pragma unroll
                for (int k = 0; k < P; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c) sm.red[g][c][li + k * BLOCK] = res[k][c];
                __syncthreads();
                if (g != 0) continue;  // group 0 adds the groups in order and stores
#pragma unroll
                for (int k = 0; k < P; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        double r = sm.red[0][c][li + k * BLOCK];
#pragma unroll
                        for (int h = 1; h < G; ++h) r += sm.red[h][c][li + k * BLOCK];
                        res[k][c] = r;
                    }
            }
            if (it.nsplit <= 1) {
#pragma unroll
                for (int k = 0; k < P; ++k)
                    if (valid[k]) subset_finalize(p, q.corr, slot[k], res[k]);
                continue;
            }
            double *mine = q.partial + (size_t)(it.pbase + it.split) * NC * CS;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int l = li + k * BLOCK;
#pragma unroll
                for (int c = 0; c < NC; ++c) mine[c * CS + l] = res[k][c];
            }
        }
    }
};

template <int BLOCK, int P, int TJ, int G, int MINB, bool EPS_ZERO>
__global__ void __launch_bounds__(BLOCK * G, MINB) subset_jerk_kernel(const F32CSubsetParams q) {
    SubsetKernel<BLOCK, P, TJ, G, EPS_ZERO>::run(q);
}

// Few-particle path (at most kFewMax active particles, F32C): every thread
// takes j-particles of the active clusters (grid-stride over their real
// particles) and evaluates them against the active particles of the same
// cluster, kFewBatch at a time; pair terms as in the subset kernel (FP32
// offsets from float-pair centres, exact centre differences, MUFU rsqrt),
// except that position differences use the offsets' low parts when given
// (q.pxl ...), so that close pairs are differenced exactly: a particle that
// steps alone is the one whose step choice the force noise would drive.
// Per thread and per warp FP32 sums, then FP64: the warps in order, the CTAs in
// a fixed order by the last CTA (ticket), which also applies the epilogue.
constexpr int kFewThreads = 256;
constexpr int kFewBatch = 6;
constexpr int kFewUnroll = 2;

__device__ void few_pass(const F32CSubsetParams &q, const int32_t *__restrict__ act, BlockScalars *sc,
                         double *__restrict__ part) {
    constexpr int nctas = kFewCtas;  // the CTAs taking part: blockIdx.x < kFewCtas
    const F32CJerkParams &p = q.base;
    __shared__ float own[kFewMax][6];
    __shared__ float ownl[kFewMax][3];  // low parts of the position offsets
    __shared__ float4 oc[kFewMax][4];
    __shared__ int ocl[kFewMax];
    __shared__ int oslot[kFewMax];  // j-set slot of each active particle (its self pair)
    __shared__ float wsum[kFewThreads / 32][kFewBatch][7];
    __shared__ double csum[kFewMax][7];
    __shared__ double fsum[kFewThreads];  // [group][output], ngrp * n_out <= kFewThreads
    __shared__ int fjb[kFewMax + 1], fab[kFewMax], fsb[kFewMax];
    __shared__ float fe2[kFewMax];
    // the corrector's inputs, fetched by cp.async while the j-loop runs: per
    // particle h, then a0, j0, v0, x0 of each component; with a mirror, its
    // tile frame (origin c0, velocity) and the frame time
    __shared__ double pre[kFewMax][13];
    __shared__ int64_t pre_u[kFewMax];
    __shared__ double pre_c0[kFewMax][3];
    __shared__ float4 pre_cv[kFewMax];
    __shared__ long long pre_t0q;
    __shared__ bool last;
    if (!sc->few) return;  // uniform: the plan chose the subset kernel
    const int na = sc->n_active;
    const int nf = sc->few_ncl;
    for (int e = threadIdx.x; e <= nf; e += blockDim.x) {
        fjb[e] = sc->few_jbase[e];
        if (e < nf) {
            const int c = sc->few_cl[e];
            fab[e] = sc->few_abeg[e];
            fsb[e] = p.cl[c].slot_begin;
            fe2[e] = p.cl[c].eps2f;
        }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < na; a += blockDim.x) {
        const int slot = act[a];
        oslot[a] = slot;
        own[a][0] = p.px[slot];
        own[a][1] = p.py[slot];
        own[a][2] = p.pz[slot];
        own[a][3] = p.pvx[slot];
        own[a][4] = p.pvy[slot];
        own[a][5] = p.pvz[slot];
        ownl[a][0] = q.pxl ? q.pxl[slot] : 0.0f;
        ownl[a][1] = q.pyl ? q.pyl[slot] : 0.0f;
        ownl[a][2] = q.pzl ? q.pzl[slot] : 0.0f;
        const int tile = slot / p.tc;
        oc[a][0] = p.chl[2 * tile];
        oc[a][1] = p.chl[2 * tile + 1];
        oc[a][2] = p.vchl[2 * tile];
        oc[a][3] = p.vchl[2 * tile + 1];
        int e = 0;
        while (e + 1 < nf && fab[e + 1] <= a) ++e;
        ocl[a] = e;  // index into the few-cluster list
        if (q.corr.sc) {
            const BlockCorrect &c = q.corr;
            const int64_t u = p.perm[slot];
            pre_u[a] = u;
            cp_async8(&pre[a][0], c.dt + u);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int64_t k = d * c.n + u;
                cp_async8(&pre[a][1 + 4 * d], c.acc + k);
                cp_async8(&pre[a][2 + 4 * d], c.jerk + k);
                cp_async8(&pre[a][3 + 4 * d], c.vel + k);
                cp_async8(&pre[a][4 + 4 * d], c.pos + k);
            }
            if (c.m.xr) {
                const int tile = slot / c.m.tc;
#pragma unroll
                for (int d = 0; d < 3; ++d) cp_async8(&pre_c0[a][d], c.m.c0 + (int64_t)d * c.m.n_tiles + tile);
                cp_async16(&pre_cv[a], c.m.vchl + 2 * tile);
                if (a == 0) cp_async8(&pre_t0q, &sc->frame_t0q);
            }
        }
    }
    cp_async_commit();
    __syncthreads();
    const int jtot = fjb[nf];
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    const int stride = nctas * kFewThreads;
    for (int b0 = 0; b0 < na; b0 += kFewBatch) {
        float acc[kFewBatch][7];
#pragma unroll
        for (int k = 0; k < kFewBatch; ++k)
#pragma unroll
            for (int c = 0; c < 7; ++c) acc[k][c] = 0.0f;
        for (int g0 = blockIdx.x * kFewThreads + threadIdx.x; g0 < jtot; g0 += kFewUnroll * stride) {
            // the loads of kFewUnroll j-particles first, so their latencies overlap
            float J[kFewUnroll][7], Jl[kFewUnroll][3];
            float4 jcen[kFewUnroll][4];
            int ej[kFewUnroll], jslot[kFewUnroll];
#pragma unroll
            for (int u = 0; u < kFewUnroll; ++u) {
                const int g = g0 + u * stride;
                ej[u] = -1;
                if (g < jtot) {
                    int e = 0;
                    while (e + 1 < nf && fjb[e + 1] <= g) ++e;
                    ej[u] = e;
                    const int js = fsb[e] + (g - fjb[e]);
                    jslot[u] = js;
                    J[u][0] = p.px[js];
                    J[u][1] = p.py[js];
                    J[u][2] = p.pz[js];
                    J[u][3] = p.pm[js];
                    J[u][4] = p.pvx[js];
                    J[u][5] = p.pvy[js];
                    J[u][6] = p.pvz[js];
                    Jl[u][0] = q.pxl ? q.pxl[js] : 0.0f;
                    Jl[u][1] = q.pyl ? q.pyl[js] : 0.0f;
                    Jl[u][2] = q.pzl ? q.pzl[js] : 0.0f;
                    const int jt = js / p.tc;
                    jcen[u][0] = p.chl[2 * jt];
                    jcen[u][1] = p.chl[2 * jt + 1];
                    jcen[u][2] = p.vchl[2 * jt];
                    jcen[u][3] = p.vchl[2 * jt + 1];
                }
            }
#pragma unroll
            for (int u = 0; u < kFewUnroll; ++u) {
                if (ej[u] < 0) continue;
                const int c = ej[u];
                const float e2 = fe2[c];
                const float jh[6] = {jcen[u][0].x, jcen[u][0].y, jcen[u][0].z,
                                     jcen[u][2].x, jcen[u][2].y, jcen[u][2].z};
                const float jl[6] = {jcen[u][1].x, jcen[u][1].y, jcen[u][1].z,
                                     jcen[u][3].x, jcen[u][3].y, jcen[u][3].z};
#pragma unroll
                for (int k = 0; k < kFewBatch; ++k) {
                    const int a = b0 + k;
                    if (a >= na || ocl[a] != c) continue;
                    const float ih[6] = {oc[a][0].x, oc[a][0].y, oc[a][0].z,
                                         oc[a][2].x, oc[a][2].y, oc[a][2].z};
                    const float il[6] = {oc[a][1].x, oc[a][1].y, oc[a][1].z,
                                         oc[a][3].x, oc[a][3].y, oc[a][3].z};
                    float r[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        float hi, lo;
                        centre_diff(ih[q], il[q], jh[q], jl[q], hi, lo);
                        if (q < 3) {
                            // positions to ~2^-48 of the offsets: with s + e =
                            // own + hi exactly (TwoSum), r = (J - s) + (Jl -
                            // (ownl + lo + e)); J - s is exact for close pairs
                            const float sm = __fadd_rn(own[a][q], hi), bb = __fsub_rn(sm, own[a][q]);
                            const float e = __fadd_rn(__fsub_rn(own[a][q], __fsub_rn(sm, bb)), __fsub_rn(hi, bb));
                            r[q] = __fadd_rn(__fsub_rn(J[u][q], sm),
                                             __fsub_rn(Jl[u][q], __fadd_rn(__fadd_rn(ownl[a][q], lo), e)));
                        } else {
                            r[q] = __fsub_rn(J[u][q + 1], __fadd_rn(__fadd_rn(own[a][q], hi), lo));
                        }
                    }
                    float r2 = __fmaf_rn(r[0], r[0], e2);
                    r2 = __fmaf_rn(r[1], r[1], r2);
                    r2 = __fmaf_rn(r[2], r[2], r2);
                    float rv = __fmul_rn(r[0], r[3]);
                    rv = __fmaf_rn(r[1], r[4], rv);
                    rv = __fmaf_rn(r[2], r[5], rv);
                    const float s = r2 > 0.0f ? rsqrt_mufu(r2) : 0.0f;
                    const float ms = __fmul_rn(J[u][3], s), s2 = __fmul_rn(s, s);
                    const float w3 = __fmul_rn(ms, s2);
                    const float beta = __fmul_rn(rv, __fmul_rn(s2, -3.0f));
                    // the self pair (r = 0 exactly) adds nothing; its potential term is masked
                    acc[k][6] = __fadd_rn(acc[k][6], jslot[u] == oslot[a] ? 0.0f : ms);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        acc[k][q] = __fmaf_rn(w3, r[q], acc[k][q]);
                        acc[k][3 + q] =
                            __fmaf_rn(w3, __fmaf_rn(beta, r[q], r[3 + q]), acc[k][3 + q]);
                    }
                }
            }
        }
        // warp trees in FP32 (no less accurate than the subset kernel's FP32
        // tile sums), then FP64: the warps in order
#pragma unroll
        for (int k = 0; k < kFewBatch; ++k) {
            if (b0 + k >= na) break;  // uniform
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                float v = acc[k][c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (lane == 0) wsum[warp][k][c] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x < kFewBatch * 7) {
            const int k = threadIdx.x / 7, c = threadIdx.x % 7;
            double v = wsum[0][k][c];
            for (int w = 1; w < kFewThreads / 32; ++w) v += wsum[w][k][c];
            if (b0 + k < na) csum[b0 + k][c] = v;
        }
        __syncthreads();
    }
    cp_async_wait_all();  // long done: the j-loop took longer (the smem is read after a barrier)
    double *mine = part + (size_t)blockIdx.x * kFewMax * 7;
    for (int t = threadIdx.x; t < na * 7; t += blockDim.x) mine[t] = csum[t / 7][t % 7];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&sc->ticket_few, 1) == nctas - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // CTA partials: output o (of na * 7) is split over ngrp thread groups, each
    // adding a fixed contiguous range of CTAs (loads issued together), then the
    // group sums are added in group order
    {
        const int n_out = na * 7;
        const int ngrp = min(kFewThreads / n_out, nctas);
        const int o = threadIdx.x % n_out, grp = threadIdx.x / n_out;
        if (grp < ngrp) {
            const int b0 = (int)((long long)grp * nctas / ngrp);
            const int b1 = (int)((long long)(grp + 1) * nctas / ngrp);
            double v = 0.0;
            for (int b = b0; b < b1; b += 8) {
                double x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    x[u] = b + u < b1 ? __ldcg(part + (size_t)(b + u) * kFewMax * 7 + o) : 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u) v += x[u];
            }
            fsum[grp * n_out + o] = v;
        }
        __syncthreads();
        if (threadIdx.x < n_out) {
            double v = fsum[threadIdx.x];
            for (int g2 = 1; g2 < ngrp; ++g2) v += fsum[g2 * n_out + threadIdx.x];
            csum[threadIdx.x / 7][threadIdx.x % 7] = v;
        }
    }
    __syncthreads();
    if (q.corr.sc) {
        // epilogue + corrector with four lanes per particle (one per
        // component, the first also for the step choice): the FP64 chain of
        // a single particle is what a small step waits for
        if (threadIdx.x < 4 * kFewMax) {
            const int a = threadIdx.x / 4, sub = threadIdx.x % 4;
            const bool valid = a < na;
            const int aa = valid ? a : 0;
            const double ph = csum[aa][6];
            const int cp = sub < 3 ? sub : 0;
            const long long tnq = sc->t_next_q;
            double fc = 0.0, fv = 0.0;
            if (q.corr.m.xr) {  // the tile frame at t_next
                fv = (double)reinterpret_cast<const float *>(&pre_cv[aa])[cp];
                fc = fma(fv, (double)(tnq - pre_t0q) * q.corr.dt_min, pre_c0[aa][cp]);
            }
            correct_particle_x4_pre<true>(q.corr, pre_u[aa], act[aa], valid, sub, pre[aa][0],
                                          pre[aa][1 + 4 * cp], pre[aa][2 + 4 * cp], pre[aa][3 + 4 * cp],
                                          pre[aa][4 + 4 * cp], fc, fv, p.G * csum[aa][cp],
                                          p.G * csum[aa][3 + cp], -p.G * ph, sc->t_next, tnq);
        }
    } else {
        for (int a = threadIdx.x; a < na; a += blockDim.x) {
            double r[7];
#pragma unroll
            for (int c = 0; c < 7; ++c) r[c] = csum[a][c];
            subset_finalize(p, q.corr, act[a], r);
        }
    }
    if (threadIdx.x == 0) sc->ticket_few = 0;
}

// Sum the partials of every i-chunk that several CTAs' ranges share, and
// finalise.  The CTAs wa..wb whose ranges cover the chunk's j-tiles follow
// from its first unit: wa wrote it to slot 2 wa if its range starts at the
// chunk, else to 2 wa + 1 (its range's last i-chunk), every later one to its
// first slot 2w.  Work unit = 32 particles of one chunk; its 8 warps each sum
// one contiguous eighth of the parts (loads unrolled, so their latencies
// overlap), then warp 0 adds the eight group sums in group order.  The order
// of every addition is fixed by the plan, so the result does not depend on
// scheduling.
constexpr int kReduceWarps = 8;

__device__ void reduce_pass(const F32CSubsetParams &q, const BlockScalars *__restrict__ sc) {
    const int cs = sc->cs;
    __shared__ double part[kReduceWarps][7][32];
    const int subs = (cs + 31) / 32;
    const int units = sc->n_chunks * subs;
    const int lane = threadIdx.x % 32, g = threadIdx.x / 32;
    const long long W = sc->n_units;
    const int nw = sc->n_workers;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        // the unit's i-chunk, its range and CTAs (every thread, the same few loads)
        const int ch = u / subs;
        int lo = 0, hi = q.ncl;
        while (hi - lo > 1) {
            const int mid = (lo + hi) / 2;
            if (q.ich_off[mid] <= ch) lo = mid;
            else hi = mid;
        }
        const int n_jt = q.base.cl[lo].n_jt, ci = ch - q.ich_off[lo];
        const long long uc = q.work_off[lo] + (long long)ci * n_jt;
        const int wa = (int)even_range_of(uc, W, nw), wb = (int)even_range_of(uc + n_jt - 1, W, nw);
        SubItem it;
        it.a0 = q.act_begin[lo] + ci * cs;
        it.na = min(cs, q.act_n[lo] - ci * cs);
        const int nparts = wb - wa + 1;
        const int l = (u % subs) * 32 + lane;
        if (nparts <= 1 || (u % subs) * 32 >= it.na) continue;  // uniform over the CTA
        // range wa's slot; every later range starts inside the chunk: slot 2r
        const int slot_a = (int)even_range_slot(wa, uc, W, nw);
        const int s0 = (int)((int64_t)g * nparts / kReduceWarps);
        const int s1 = (int)((int64_t)(g + 1) * nparts / kReduceWarps);
        double tot[7] = {0, 0, 0, 0, 0, 0, 0};
        if (l < it.na) {
#pragma unroll 4
            for (int s = s0; s < s1; ++s) {
                const double *ps = q.partial + (size_t)(s == 0 ? slot_a : 2 * (wa + s)) * 7 * cs + l;
#pragma unroll
                for (int c = 0; c < 7; ++c) tot[c] += ps[c * cs];
            }
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) part[g][c][lane] = tot[c];
        __syncthreads();
        if (q.corr.sc) {
            // the unit's 32 particles corrected four lanes each (one per
            // component): the FP64 chain of one particle is what a step of a
            // few chunks waits for
            if (threadIdx.x < 4 * 32) {
                const int a = threadIdx.x / 4, sub = threadIdx.x % 4, cp = sub < 3 ? sub : 0;
                const int la = (u % subs) * 32 + a;
                const bool valid = la < it.na;
                double ra = part[0][cp][a], rj = part[0][3 + cp][a], rp = part[0][6][a];
#pragma unroll
                for (int h = 1; h < kReduceWarps; ++h) {
                    ra += part[h][cp][a];
                    rj += part[h][3 + cp][a];
                    rp += part[h][6][a];
                }
                const int slot = q.act_slot[it.a0 + (valid ? la : (u % subs) * 32)];
                const double G = q.base.G;
                correct_particle_x4<true>(q.corr, q.base.perm[slot], slot, valid, sub, G * ra, G * rj, -G * rp,
                                          sc->t_next, sc->t_next_q);
            }
        } else if (g == 0 && l < it.na) {
            double r[7];
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                r[c] = part[0][c][lane];
#pragma unroll
                for (int h = 1; h < kReduceWarps; ++h) r[c] += part[h][c][lane];
            }
            subset_finalize(q.base, q.corr, q.act_slot[it.a0 + l], r);
        }
        __syncthreads();
    }
}

// The force pass's last kernel: the few-particle pass when the plan chose it
// (on kFewCtas CTAs), else the ordered sum of the shared i-chunks' partials.
// One launch for either, after the subset kernels (which have no work in the
// few-particle case).
static_assert(kFewThreads == 32 * kReduceWarps, "one block size for both passes");

__global__ void __launch_bounds__(kFewThreads, 2)
    subset_tail_kernel(const F32CSubsetParams q, const int32_t *__restrict__ act, BlockScalars *sc,
                       double *__restrict__ few_part) {
    if (sc->few) {  // uniform
        if ((int)blockIdx.x < kFewCtas) few_pass(q, act, sc, few_part);
        return;
    }
    reduce_pass(q, sc);
}

struct SubsetShape {
    int block, p, tj, groups, minb;
    bool eps_zero;
    const void *kernel;
};

#define SUBSET(B, P, T, G, M)                                                                    \
    SubsetShape{B, P, T, G, M, false, (const void *)subset_jerk_kernel<B, P, T, G, M, false>},   \
        SubsetShape{B, P, T, G, M, true, (const void *)subset_jerk_kernel<B, P, T, G, M, true>}

// Small active sets: several thread groups per CTA split each j-tile (more
// warps on few i-chunks); large ones: one group, P = 2 (more reuse per load).
const SubsetShape kSubsetShapes[] = {SUBSET(64, 1, 256, 4, 2), SUBSET(64, 1, 128, 4, 2),
                                     SUBSET(64, 1, 512, 4, 2), SUBSET(64, 2, 256, 1, 4),
                                     SUBSET(64, 2, 128, 1, 4), SUBSET(64, 2, 512, 1, 4)};

const SubsetShape *find_subset(int block, int p, int tj, int groups, int minb, bool eps_zero) {
    for (const SubsetShape &s : kSubsetShapes)
        if (s.block == block && s.p == p && s.tj == tj && s.groups == groups && s.minb == minb &&
            s.eps_zero == eps_zero)
            return &s;
    return nullptr;
}

// FP64 subset kernel: one CTA per active chunk (of kF64Block particles), each
// thread one active particle against every predicted particle of its cluster.
__global__ void __launch_bounds__(kF64Block)
    subset_f64_kernel(const double *__restrict__ xp, const double *__restrict__ vp,
                      const double *__restrict__ mass, const ClusterDev *__restrict__ cls,
                      const SubItem *__restrict__ items, const int *__restrict__ n_items,
                      const int32_t *__restrict__ act, int64_t n, double G, double *acc,
                      double *jerk, double *pot) {
    if ((int)blockIdx.x >= *n_items) return;
    __shared__ double sj[7][kF64Block];
    const SubItem it = items[blockIdx.x];
    const ClusterDev cl = cls[it.cluster];
    const bool valid = (int)threadIdx.x < it.na;
    const int64_t i = act[it.a0 + (valid ? threadIdx.x : 0)];
    const double xi = xp[i], yi = xp[n + i], zi = xp[2 * n + i];
    const double ui = vp[i], vi = vp[n + i], wi = vp[2 * n + i];
    double s7[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int j0 = 0; j0 < cl.n; j0 += kF64Block) {
        const int lj = j0 + threadIdx.x;
        __syncthreads();
        if (lj < cl.n) {
            const int64_t j = cl.user_begin + lj;
            sj[0][threadIdx.x] = xp[j];
            sj[1][threadIdx.x] = xp[n + j];
            sj[2][threadIdx.x] = xp[2 * n + j];
            sj[3][threadIdx.x] = mass[j];
            sj[4][threadIdx.x] = vp[j];
            sj[5][threadIdx.x] = vp[n + j];
            sj[6][threadIdx.x] = vp[2 * n + j];
        }
        __syncthreads();
        const int cnt = min(kF64Block, cl.n - j0);
        for (int k = 0; k < cnt; ++k) {
            const double dx = sj[0][k] - xi, dy = sj[1][k] - yi, dz = sj[2][k] - zi;
            const double ux = sj[4][k] - ui, uy = sj[5][k] - vi, uz = sj[6][k] - wi;
            const double r2 = dx * dx + dy * dy + dz * dz + cl.eps2;
            const bool skip = (cl.user_begin + j0 + k == i) || !(r2 > 0.0);
            const double s = skip ? 0.0 : rsqrt(r2);
            const double ms = sj[3][k] * s, s2 = s * s, w3 = ms * s2;
            const double beta = -3.0 * (dx * ux + dy * uy + dz * uz) * s2;
            s7[6] += ms;
            s7[0] += w3 * dx;
            s7[1] += w3 * dy;
            s7[2] += w3 * dz;
            s7[3] += w3 * (ux + beta * dx);
            s7[4] += w3 * (uy + beta * dy);
            s7[5] += w3 * (uz + beta * dz);
        }
    }
    if (!valid) return;
    for (int d = 0; d < 3; ++d) {
        acc[d * n + i] = G * s7[d];
        jerk[d * n + i] = G * s7[3 + d];
    }
    pot[i] = -G * s7[6];
}

}  // namespace

int subset_shapes(int *block, int *p, int *tj, int *groups, int *minb, int cap) {
    int n = 0;
    for (const SubsetShape &s : kSubsetShapes) {
        if (s.eps_zero) continue;
        if (n < cap) {
            block[n] = s.block;
            p[n] = s.p;
            tj[n] = s.tj;
            groups[n] = s.groups;
            minb[n] = s.minb;
        }
        ++n;
    }
    return n;
}

cudaError_t launch_subset_tail(int max_chunks, int max_cs, int max_ctas, const F32CSubsetParams &prm,
                               const int32_t *act, BlockScalars *sc, double *few_part, cudaStream_t s) {
    const int64_t units = (int64_t)max_chunks * ((max_cs + 31) / 32);
    const int grid = (int)std::max<int64_t>(kFewCtas, std::min<int64_t>(units, max_ctas));
    subset_tail_kernel<<<grid, kFewThreads, 0, s>>>(prm, act, sc, few_part);
    return cudaGetLastError();
}

int subset_occupancy(int block, int p, int tj, int groups, int minb, bool eps_zero) {
    const SubsetShape *s = find_subset(block, p, tj, groups, minb, eps_zero);
    if (!s) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, s->kernel, block * groups, 0) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_subset_f32c(int block, int p, int tj, int groups, int minb, bool eps_zero,
                               int grid, const F32CSubsetParams &prm, cudaStream_t st) {
    const SubsetShape *sh = find_subset(block, p, tj, groups, minb, eps_zero);
    if (!sh) return cudaErrorNotSupported;
    if (grid <= 0) return cudaSuccess;
    void *args[] = {(void *)&prm};
    return cudaLaunchKernel(sh->kernel, dim3(grid), dim3(block * groups), args, 0, st);
}

cudaError_t launch_subset_f64(int max_items, const double *xp, const double *vp, const double *mass,
                              const ClusterDev *cl, const SubItem *items, const int *n_items,
                              const int32_t *act, int64_t n, double G, double *acc, double *jerk,
                              double *pot, cudaStream_t s) {
    if (max_items <= 0) return cudaSuccess;
    subset_f64_kernel<<<max_items, kF64Block, 0, s>>>(xp, vp, mass, cl, items, n_items, act, n, G, acc,
                                                     jerk, pot);
    return cudaGetLastError();
}

}  // namespace nbody
