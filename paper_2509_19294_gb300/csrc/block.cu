// block.cu -- individual (block) time steps: scheduling and forces on the
// active subset.
//
// Around the Hermite scheme each particle keeps its own time t_i and a
// power-of-two step dt_i (Makino & Aarseth 1992; the paper computes the jerk,
// Sec. 3, but does not describe its stepping).  One block step, all on the
// device so that it is a fixed kernel sequence a CUDA graph can replay
// (F32C; the FP64 path keeps separate predict / count / plan / scatter /
// items / correct kernels around its own subset kernel):
//   1. block_min_kernel: t_next = min_i (t_i + dt_i), an integer min in units
//      of dt_min (exact)
//   2. block_pack_kernel: predict every particle to t_next, pack it as the
//      j-set (the jerk path's geometry), flag and count the active slots per
//      tile; the last CTA plans the step (offsets, regime, split, queue size)
//   3. block_queue_kernel: ordered compaction of the active slots, work items
//   4. the force pass: the small-set and the large-set subset kernels, then
//      subset_tail_kernel, which either runs the few-particle pass (<= kFewMax
//      active; the subset kernels then find an empty queue) or sums the
//      subset kernels' split partials in order
//   5. the Hermite corrector and next-step choice, in the epilogue of 4
// An active particle is evaluated with its own j-set offset and its own tile
// centre: per j-tile each thread forms the exact centre difference for each of
// its particles, so the self pair is exactly zero, as in the full kernels.
#include <algorithm>
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "block_reduce.cuh"
#include "forces_f32c_jerk.cuh"
#include "nbody_internal.h"

namespace nbody {

namespace {

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
// an integer test in units of dt_min).  Records the particle's new time, step
// and level.
__device__ __forceinline__ void choose_step(const BlockCorrect &c, int64_t i, double h, double na,
                                            double nj, double n2, double n3, double tn, long long tnq) {
    const double den = nj * n3 + n2 * n2;
    const double da = den > 0.0 ? sqrt(c.eta * (na * n2 + nj * nj) / den) : c.dt_max;
    const double inv_dt_min = recip_pow2(c.dt_min);
    double nd = h;
    while (nd > da && nd > c.dt_min) nd *= 0.5;
    const long long q2 = (long long)(2.0 * h * inv_dt_min);  // 2h in units of dt_min
    if (nd == h && da >= 2.0 * h && 2.0 * h <= c.dt_max && tnq % q2 == 0) nd = 2.0 * h;
    if (c.level && nd != h) {
        atomicSub(&c.level[block_level(h, c.dt_max)], 1);
        atomicAdd(&c.level[block_level(nd, c.dt_max)], 1);
    }
    c.t[i] = tn;
    c.dt[i] = nd;
    c.tq[i] = tnq + (long long)(nd * inv_dt_min);
}

// Hermite corrector of active particle (row) i over its step h = dt_i with the
// new acceleration A1, jerk J1 and potential p1, then its next step by
// Aarseth's criterion.  Steps are powers of two >= dt_min and t_next is a
// multiple of dt_min, so dividing by h, h^2, h^3 is the exact multiplication
// by their reciprocals and "t_next is a multiple of 2h" is an integer test;
// both give the oracle's results bit for bit.
__device__ __forceinline__ void correct_particle(const BlockCorrect &c, int64_t i, const double (&A1)[3],
                                                 const double (&J1)[3], double p1, double tn,
                                                 long long tnq) {
    const double h = c.dt[i], h2 = h * h;
    const double ih = recip_pow2(h), ih2 = ih * ih, ih3 = ih2 * ih;
    double A2[3], A3[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int64_t q = d * c.n + i;
        const double a0 = c.acc[q], j0 = c.jerk[q], v0 = c.vel[q];
        const double v1 = v0 + (a0 + A1[d]) * h / 2.0 + (j0 - J1[d]) * h2 / 12.0;
        c.pos[q] = c.pos[q] + (v0 + v1) * h / 2.0 + (a0 - A1[d]) * h2 / 12.0;
        c.vel[q] = v1;
        A3[d] = (12.0 * (a0 - A1[d]) + 6.0 * h * (j0 + J1[d])) * ih3;
        A2[d] = (-6.0 * (a0 - A1[d]) - h * (4.0 * j0 + 2.0 * J1[d])) * ih2 + h * A3[d];
        c.acc[q] = A1[d];
        c.jerk[q] = J1[d];
        if (c.af) {
            c.af[q] = (float)A1[d];
            c.jf[q] = (float)J1[d];
        }
    }
    if (c.pot) c.pot[i] = p1;
    const double na = sqrt(A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2]);
    const double nj = sqrt(J1[0] * J1[0] + J1[1] * J1[1] + J1[2] * J1[2]);
    const double n2 = sqrt(A2[0] * A2[0] + A2[1] * A2[1] + A2[2] * A2[2]);
    const double n3 = sqrt(A3[0] * A3[0] + A3[1] * A3[1] + A3[2] * A3[2]);
    choose_step(c, i, h, na, nj, n2, n3, tn, tnq);
}

// correct_particle spread over four consecutive lanes of a warp: lane sub
// (0..2) corrects component sub, the norms are summed across the three lanes
// in component order, and lane 0 chooses the step.  Every lane of the warp
// calls it (the shuffles need them); lanes with valid == false store nothing.
__device__ __forceinline__ void correct_particle_x4(const BlockCorrect &c, int64_t i, bool valid, int sub,
                                                    double a1, double j1, double p1, double tn,
                                                    long long tnq) {
    const double h = c.dt[i], h2 = h * h;
    const double ih = recip_pow2(h), ih2 = ih * ih, ih3 = ih2 * ih;
    double sq[4] = {0.0, 0.0, 0.0, 0.0};  // this component's a1^2, j1^2, a2^2, a3^2
    if (sub < 3) {
        const int64_t q = sub * c.n + i;
        const double a0 = c.acc[q], j0 = c.jerk[q], v0 = c.vel[q];
        const double v1 = v0 + (a0 + a1) * h / 2.0 + (j0 - j1) * h2 / 12.0;
        const double x1 = c.pos[q] + (v0 + v1) * h / 2.0 + (a0 - a1) * h2 / 12.0;
        const double a3 = (12.0 * (a0 - a1) + 6.0 * h * (j0 + j1)) * ih3;
        const double a2 = (-6.0 * (a0 - a1) - h * (4.0 * j0 + 2.0 * j1)) * ih2 + h * a3;
        if (valid) {
            c.pos[q] = x1;
            c.vel[q] = v1;
            c.acc[q] = a1;
            c.jerk[q] = j1;
            if (c.af) {
                c.af[q] = (float)a1;
                c.jf[q] = (float)j1;
            }
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
        nrm[k] = sqrt(x + y + z);
    }
    if (sub != 0 || !valid) return;
    if (c.pot) c.pot[i] = p1;
    choose_step(c, i, h, nrm[0], nrm[1], nrm[2], nrm[3], tn, tnq);
}

// FP64 epilogue of one active particle: scale by G, remove the self term of
// phi (its own j-tile contributed m_i rsqrt(eps^2) exactly), then correct the
// particle (corr.sc set) or store a1, j1, p1 at its row.
__device__ __forceinline__ void subset_finalize(const F32CJerkParams &p, const BlockCorrect &corr,
                                                const ClusterDev &cl, int slot, const double (&r)[7]) {
    const int64_t u = p.perm[slot];
    double ph = r[6];
    if (cl.eps2f > 0.0f) ph -= (double)__fmul_rn(p.pm[slot], rsqrt_mufu(cl.eps2f));
    if (corr.sc) {
        const double A1[3] = {p.G * r[0], p.G * r[1], p.G * r[2]};
        const double J1[3] = {p.G * r[3], p.G * r[4], p.G * r[5]};
        correct_particle(corr, u, A1, J1, -p.G * ph, corr.sc->t_next, corr.sc->t_next_q);
        return;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p.acc[d * p.n + u] = p.G * r[d];
        p.jerk[d * p.n + u] = p.G * r[3 + d];
    }
    if (p.pot) p.pot[u] = -p.G * ph;
}

// Subset kernel: persistent CTAs over the device-built queue of (i-chunk of the
// active list, j-range) items.  A CTA holds BLOCK * P active particles (P per
// thread) in G thread groups of BLOCK; all groups hold the same particles and
// each takes one G-th of every shared-memory j-tile, so a small active set
// still keeps G times more warps busy.  The groups' Kahan sums are added in
// group order (FP64, shared memory); a j-range split is written as an FP64
// partial that subset_tail_kernel sums in split order.
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
        const int n_items = *q.n_items;
        // CTAs beyond the item count would find the queue empty: they leave
        // without touching its head (the others still drain it)
        if ((int)blockIdx.x >= n_items) return;
        const int li = threadIdx.x % BLOCK, g = threadIdx.x / BLOCK;
        for (;;) {
            if (threadIdx.x == 0) sm.item = atomicAdd(p.counters, 1);
            __syncthreads();
            const int item_idx = sm.item;
            if (item_idx >= n_items) break;
            const SubItem it = q.items[item_idx];
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
#pragma unroll 1
                for (int v = g * COLS; v < (g + 1) * COLS; ++v) {
                    float4 Q[NA];
#pragma unroll
                    for (int a = 0; a < NA; ++a) Q[a] = sm.j[b][a][v];
                    float2 J[NA];
#pragma unroll
                    for (int a = 0; a < NA; ++a) J[a] = make_float2(Q[a].x, Q[a].y);
                    JK::body(J, e2, ni, acc);
#pragma unroll
                    for (int a = 0; a < NA; ++a) J[a] = make_float2(Q[a].z, Q[a].w);
                    JK::body(J, e2, ni, acc);
                }
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
                    if (valid[k]) subset_finalize(p, q.corr, cl, slot[k], res[k]);
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
// offsets from float-pair centres, exact centre differences, MUFU rsqrt).
// Per thread and per warp FP32 sums, then FP64: the warps in order, the CTAs in
// a fixed order by the last CTA (ticket), which also applies the epilogue.
constexpr int kFewThreads = 256;
constexpr int kFewBatch = 8;
constexpr int kFewUnroll = 2;

__device__ void few_pass(const F32CSubsetParams &q, const int32_t *__restrict__ act, BlockScalars *sc,
                         double *__restrict__ part) {
    constexpr int nctas = kFewCtas;  // the CTAs taking part: blockIdx.x < kFewCtas
    const F32CJerkParams &p = q.base;
    __shared__ float own[kFewMax][6];
    __shared__ float4 oc[kFewMax][4];
    __shared__ int ocl[kFewMax];
    __shared__ float wsum[kFewThreads / 32][kFewBatch][7];
    __shared__ double csum[kFewMax][7];
    __shared__ double fsum[kFewThreads];  // [group][output], ngrp * n_out <= kFewThreads
    __shared__ int fjb[kFewMax + 1], fcl[kFewMax], fab[kFewMax], fsb[kFewMax];
    __shared__ float fe2[kFewMax];
    __shared__ bool last;
    if (!sc->few) return;  // uniform: the plan chose the subset kernel
    const int na = sc->n_active;
    const int nf = sc->few_ncl;
    for (int e = threadIdx.x; e <= nf; e += blockDim.x) {
        fjb[e] = sc->few_jbase[e];
        if (e < nf) {
            const int c = sc->few_cl[e];
            fcl[e] = c;
            fab[e] = sc->few_abeg[e];
            fsb[e] = p.cl[c].slot_begin;
            fe2[e] = p.cl[c].eps2f;
        }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < na; a += blockDim.x) {
        const int slot = act[a];
        own[a][0] = p.px[slot];
        own[a][1] = p.py[slot];
        own[a][2] = p.pz[slot];
        own[a][3] = p.pvx[slot];
        own[a][4] = p.pvy[slot];
        own[a][5] = p.pvz[slot];
        const int tile = slot / p.tc;
        oc[a][0] = p.chl[2 * tile];
        oc[a][1] = p.chl[2 * tile + 1];
        oc[a][2] = p.vchl[2 * tile];
        oc[a][3] = p.vchl[2 * tile + 1];
        int e = 0;
        while (e + 1 < nf && fab[e + 1] <= a) ++e;
        ocl[a] = e;  // index into the few-cluster list
    }
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
            float J[kFewUnroll][7];
            float4 jcen[kFewUnroll][4];
            int ej[kFewUnroll];
#pragma unroll
            for (int u = 0; u < kFewUnroll; ++u) {
                const int g = g0 + u * stride;
                ej[u] = -1;
                if (g < jtot) {
                    int e = 0;
                    while (e + 1 < nf && fjb[e + 1] <= g) ++e;
                    ej[u] = e;
                    const int js = fsb[e] + (g - fjb[e]);
                    J[u][0] = p.px[js];
                    J[u][1] = p.py[js];
                    J[u][2] = p.pz[js];
                    J[u][3] = p.pm[js];
                    J[u][4] = p.pvx[js];
                    J[u][5] = p.pvy[js];
                    J[u][6] = p.pvz[js];
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
                        r[q] = __fsub_rn(J[u][q < 3 ? q : q + 1],
                                         __fadd_rn(__fadd_rn(own[a][q], hi), lo));
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
                    acc[k][6] = __fadd_rn(acc[k][6], ms);
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
            const ClusterDev cl = p.cl[fcl[ocl[aa]]];
            const int slot = act[aa];
            double ph = csum[aa][6];
            if (cl.eps2f > 0.0f) ph -= (double)__fmul_rn(p.pm[slot], rsqrt_mufu(cl.eps2f));
            correct_particle_x4(q.corr, p.perm[slot], valid, sub, p.G * csum[aa][sub < 3 ? sub : 0],
                                p.G * csum[aa][sub < 3 ? 3 + sub : 3], -p.G * ph, sc->t_next,
                                sc->t_next_q);
        }
    } else {
        for (int a = threadIdx.x; a < na; a += blockDim.x) {
            double r[7];
#pragma unroll
            for (int c = 0; c < 7; ++c) r[c] = csum[a][c];
            subset_finalize(p, q.corr, p.cl[fcl[ocl[a]]], act[a], r);
        }
    }
    if (threadIdx.x == 0) sc->ticket_few = 0;
}

// Sum the split partials of every chunk and finalise.  Work unit = 32
// particles of one chunk; its 8 warps each sum one contiguous eighth of the
// splits (loads unrolled, so their latencies overlap), then warp 0 adds the
// eight group sums in group order.  The order of every addition is fixed by
// (nsplit, particle), so the result does not depend on scheduling.
constexpr int kReduceWarps = 8;

__device__ void reduce_pass(const F32CSubsetParams &q, const SubItem *__restrict__ info,
                            const BlockScalars *__restrict__ sc) {
    const int cs = sc->cs;
    __shared__ double part[kReduceWarps][7][32];
    const int subs = (cs + 31) / 32;
    const int units = sc->n_chunks * subs;
    const int lane = threadIdx.x % 32, g = threadIdx.x / 32;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const SubItem it = info[u / subs];
        const int l = (u % subs) * 32 + lane;
        if (it.nsplit <= 1 || (u % subs) * 32 >= it.na) continue;  // uniform over the CTA
        const int s0 = (int)((int64_t)g * it.nsplit / kReduceWarps);
        const int s1 = (int)((int64_t)(g + 1) * it.nsplit / kReduceWarps);
        double tot[7] = {0, 0, 0, 0, 0, 0, 0};
        if (l < it.na) {
#pragma unroll 4
            for (int s = s0; s < s1; ++s) {
                const double *ps = q.partial + (size_t)(it.pbase + s) * 7 * cs + l;
#pragma unroll
                for (int c = 0; c < 7; ++c) tot[c] += ps[c * cs];
            }
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) part[g][c][lane] = tot[c];
        __syncthreads();
        if (g == 0 && l < it.na) {
            double r[7];
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                r[c] = part[0][c][lane];
#pragma unroll
                for (int h = 1; h < kReduceWarps; ++h) r[c] += part[h][c][lane];
            }
            subset_finalize(q.base, q.corr, q.base.cl[it.cluster], q.act_slot[it.a0 + l], r);
        }
        __syncthreads();
    }
}

// The force pass's last kernel: the few-particle pass when the plan chose it
// (on kFewCtas CTAs), else the ordered sum of the subset kernels' split
// partials.  One launch for either, after the subset kernels (which find an
// empty queue in the few-particle case).
static_assert(kFewThreads == 32 * kReduceWarps, "one block size for both passes");

__global__ void __launch_bounds__(kFewThreads)
    subset_tail_kernel(const F32CSubsetParams q, const int32_t *__restrict__ act, BlockScalars *sc,
                       double *__restrict__ few_part, const SubItem *__restrict__ info) {
    if (sc->few) {  // uniform
        if ((int)blockIdx.x < kFewCtas) few_pass(q, act, sc, few_part);
        return;
    }
    reduce_pass(q, info, sc);
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

constexpr int kScan = 1024;

// Initial steps: the largest power of two <= min(dt_max, eta_s |a| / |j|), >= dt_min.
__global__ void block_init_kernel(int64_t n, const double *acc, const double *jerk, double dt_max,
                                  double dt_min, double eta_s, double *t, double *dt, long long *tq) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double an = sqrt(acc[i] * acc[i] + acc[n + i] * acc[n + i] + acc[2 * n + i] * acc[2 * n + i]);
        const double jn =
            sqrt(jerk[i] * jerk[i] + jerk[n + i] * jerk[n + i] + jerk[2 * n + i] * jerk[2 * n + i]);
        double d = jn > 0.0 ? eta_s * an / jn : dt_max;
        if (!(d < dt_max)) d = dt_max;
        d = exp2(floor(log2(d)));
        if (d < dt_min) d = dt_min;
        t[i] = 0.0;
        dt[i] = d;
        tq[i] = (long long)(d / dt_min);
    }
}

// FP32 copies of a and a' for the packing predictor (start of block stepping).
__global__ void block_shadow_kernel(int64_t n3, const double *__restrict__ acc,
                                    const double *__restrict__ jerk, float *af, float *jf) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3;
         k += (int64_t)gridDim.x * blockDim.x) {
        af[k] = (float)acc[k];
        jf[k] = (float)jerk[k];
    }
}

// Count the particles per step level (start of block stepping).
__global__ void block_levels_kernel(int64_t n, const double *__restrict__ dt, double dt_max,
                                    BlockScalars *sc) {
    __shared__ int cnt[64];
    for (int k = threadIdx.x; k < 64; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[block_level(dt[i], dt_max)], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < 64; k += blockDim.x)
        if (cnt[k]) atomicAdd(&sc->level[k], cnt[k]);
}

// t_next = min_i (t_i + dt_i), exact: the times are integers in units of
// dt_min, so the min is an integer one.  Per-chunk minima, then the last CTA
// to finish (ticket) takes the min over them.  No CTA waits for another.
constexpr int kMinThreads = 512;

__global__ void __launch_bounds__(kMinThreads)
    block_min_kernel(const long long *__restrict__ tq, const Chunk *__restrict__ chunks,
                     long long *__restrict__ part, int n_chunks, double dt_min, BlockScalars *sc) {
    __shared__ long long red[kMinThreads / 32];
    __shared__ bool last;
    const Chunk ch = chunks[blockIdx.x];
    long long m = LLONG_MAX;
    for (int64_t i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) m = min(m, tq[i]);
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kMinThreads / 32; ++w) m = min(m, red[w]);
        part[blockIdx.x] = m;
        __threadfence();
        last = atomicAdd(&sc->ticket_min, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    m = LLONG_MAX;
    for (int k = threadIdx.x; k < n_chunks; k += blockDim.x) m = min(m, __ldcg(part + k));
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kMinThreads / 32; ++w) m = min(m, red[w]);
        sc->t_next_q = m;
        sc->t_next = (double)m * dt_min;
        sc->ticket_min = 0;
    }
}

// Hermite predictor of particle (row) u to time tn: x[0..2] position, x[3..5] velocity.
__device__ __forceinline__ void predict_row(int64_t n, int64_t u, double tn, const double *__restrict__ t,
                                            const double *__restrict__ pos, const double *__restrict__ vel,
                                            const double *__restrict__ acc,
                                            const double *__restrict__ jerk, double (&x)[6]) {
    const double h = tn - t[u], h2 = h * h, h3 = h2 * h;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int64_t q = d * n + u;
        x[d] = pos[q] + vel[q] * h + acc[q] * h2 / 2.0 + jerk[q] * h3 / 6.0;
        x[3 + d] = vel[q] + acc[q] * h + jerk[q] * h2 / 2.0;
    }
}

// Predict every particle to t_next and flag the active ones (FP64 path).
__global__ void block_predict_kernel(int64_t n, const BlockScalars *__restrict__ sc,
                                     const double *__restrict__ t,
                                     const long long *__restrict__ tq, const double *__restrict__ pos,
                                     const double *__restrict__ vel, const double *__restrict__ acc,
                                     const double *__restrict__ jerk, double *xp, double *vp,
                                     uint8_t *flag) {
    const double tn = sc->t_next;
    const bool live = tn <= sc->t_end;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x[6];
        predict_row(n, i, tn, t, pos, vel, acc, jerk, x);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xp[d * n + i] = x[d];
            vp[d * n + i] = x[3 + d];
        }
        flag[i] = live && tq[i] == sc->t_next_q;
    }
}

// Compaction stage 1 (FP64 path): active count per chunk.
__global__ void block_count_kernel(const uint8_t *__restrict__ flag, const Chunk *__restrict__ chunks,
                                   int *__restrict__ cnt) {
    __shared__ int red[8];
    const Chunk ch = chunks[blockIdx.x];
    int c = 0;
    for (int64_t i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) c += flag[i];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) c += red[w];
        cnt[blockIdx.x] = c;
    }
}

// Block-wide exclusive scan of int values by a CTA of NT threads (L2 reads, so
// the last CTA of a kernel sees what the others wrote).
template <int NT>
__device__ void block_exclusive_scan(const int *in, int *out, int n, int *total) {
    __shared__ int warp_sums[NT / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += NT) {
        const int i = base + threadIdx.x;
        const int v = i < n ? __ldcg(in + i) : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x % 32) >= o) x += y;
        }
        if (threadIdx.x % 32 == 31) warp_sums[threadIdx.x / 32] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int w = threadIdx.x < NT / 32 ? warp_sums[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (threadIdx.x >= o) w += y;
            }
            if (threadIdx.x < NT / 32) warp_sums[threadIdx.x] = w;
        }
        __syncthreads();
        const int warp_off = threadIdx.x >= 32 ? warp_sums[threadIdx.x / 32 - 1] : 0;
        if (i < n) out[i] = carry + warp_off + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[NT / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// The step's plan (one thread, after the scan of the per-unit active counts;
// cluster c owns units [unit_first[c], unit_first[c + 1])): per-cluster active
// ranges and i-chunk counts, the split count, the work-queue size, and the
// queue head reset for the subset kernel.
__device__ void plan_step(const int *__restrict__ unit_off, int total, int n_units,
                          const int32_t *__restrict__ unit_first, int ncl,
                          const ClusterDev *__restrict__ cl, int cs_small, int workers_small,
                          int max_split, int *__restrict__ act_begin, int *__restrict__ act_n,
                          int *__restrict__ ich_off, int *__restrict__ item_off, BlockScalars *sc,
                          int *queue_head, int few_max, int cs_large, int workers_large, int large_min,
                          long long partial_cap) {
    const bool few = total > 0 && total <= few_max;
    const bool large = !few && cs_large > 0 && total >= large_min;
    const int cs = large ? cs_large : cs_small;
    const int workers = large ? workers_large : workers_small;
    int chunks = 0, nf = 0, jb = 0;
    for (int c = 0; c < ncl; ++c) {
        const int b = unit_first[c], e = unit_first[c + 1];
        const int a0 = b < n_units ? unit_off[b] : total;
        const int a1 = e < n_units ? unit_off[e] : total;
        act_begin[c] = a0;
        act_n[c] = a1 - a0;
        ich_off[c] = chunks;
        if (!few) chunks += (a1 - a0 + cs - 1) / cs;
        if (few && a1 > a0) {  // at most total (<= kFewMax) clusters
            sc->few_cl[nf] = c;
            sc->few_abeg[nf] = a0;
            sc->few_jbase[nf] = jb;
            jb += cl[c].n;
            ++nf;
        }
    }
    ich_off[ncl] = chunks;
    sc->few = few;
    sc->few_ncl = nf;
    sc->few_jbase[nf] = jb;
    int split = chunks > 0 ? (2 * workers) / chunks : 1;
    if (split > max_split) split = max_split;
    if (split < 1) split = 1;
    // equal-cost items drain in ceil(items / workers) rounds: among the next few
    // split counts that fit the partial buffer, take the one whose last round
    // is fullest (the smaller on ties)
    if (chunks > 0) {
        const long long max_slots = partial_cap / (7LL * cs);
        double best = -1.0;
        int pick = split;
        for (int sp = split; sp <= split + 3 && sp <= max_split; ++sp) {
            if (sp > 1 && (long long)chunks * sp > max_slots) break;
            const double r = (double)chunks * sp / workers;
            const double eff = r / ceil(r);
            if (eff > best + 1e-9) {
                best = eff;
                pick = sp;
            }
        }
        split = pick;
    }
    int items = 0;
    for (int c = 0; c < ncl; ++c) {
        item_off[c] = items;
        const int sc_c = split < cl[c].n_jt ? split : (cl[c].n_jt > 0 ? cl[c].n_jt : 1);
        items += (ich_off[c + 1] - ich_off[c]) * sc_c;
    }
    item_off[ncl] = items;
    sc->n_active = total;
    sc->n_chunks = chunks;
    sc->split = split;
    sc->n_items = items;
    sc->cs = cs;
    sc->n_items_small = large ? 0 : items;
    sc->n_items_large = large ? items : 0;
    if (total > 0) {
        sc->blocks += 1;
        sc->evals += total;
    }
    if (queue_head) queue_head[0] = queue_head[1] = 0;  // small and large subset kernels
}

// Compaction stage 2 (FP64 path, one CTA): chunk offsets and the plan.
__global__ void __launch_bounds__(kScan)
    block_plan_kernel(const int *__restrict__ cnt, int n_chunks, const int32_t *__restrict__ chunk_first,
                      int ncl, const ClusterDev *__restrict__ cl, int cs, int workers, int max_split,
                      int *__restrict__ chunk_off, int *__restrict__ act_begin, int *__restrict__ act_n,
                      int *__restrict__ ich_off, int *__restrict__ item_off, BlockScalars *sc) {
    __shared__ int total;
    block_exclusive_scan<kScan>(cnt, chunk_off, n_chunks, &total);
    __syncthreads();
    if (threadIdx.x == 0)
        plan_step(chunk_off, total, n_chunks, chunk_first, ncl, cl, cs, workers, max_split, act_begin,
                  act_n, ich_off, item_off, sc, nullptr, 0, 0, 0, 0, 0);
}

// F32C: one CTA per centre tile of the j-set.  Predicts the tile's particles to
// t_next (FP64, as block_predict_kernel), packs them as pack_kernel does
// (FP64 mean position and velocity as float pairs, FP32 offsets, FP32 masses,
// pads far away with mass 0), flags the active slots and counts them.  The
// last CTA to finish (ticket) scans the tile counts and plans the step.
struct BlockPackParams {
    const int32_t *perm;
    const ClusterDev *cl;
    const int32_t *tile_cluster;
    int tc, n_tiles;
    int64_t n;
    const double *mass, *t, *pos, *vel;
    const float *af, *jf;  // FP32 copies of each particle's a, a' (kept by the corrector)
    const long long *tq;
    float *px, *py, *pz, *pm, *pvx, *pvy, *pvz;
    float4 *chl, *vchl;
    uint8_t *flag;  // per slot
    int *tile_cnt, *tile_off;
    const int32_t *tile_first;
    int ncl, cs, workers, max_split;
    int *act_begin, *act_n, *ich_off, *item_off;
    BlockScalars *sc;
    int *queue_head;
    int few_max;
    int cs_large, workers_large, large_min;
    long long partial_cap;  // doubles in the split-partial buffer
    double dt_max, dt_min;
};

// Hermite predictor for the packed j-set (F32C): x + h v in FP64, the
// higher-order terms h^2 (a/2 + h a'/6) and h (a + h a'/2) in FP32 from FP32
// copies of a and a'.  They are small against the step's displacement, so
// their FP32 rounding stays far below that of the packed FP32 offsets; FP64
// operations, scarce on this part, drop from 24 to 11 per particle (the
// velocity change is returned apart, for the packed offset).
__device__ __forceinline__ void predict_mixed(const BlockPackParams &q, int64_t u, double tn,
                                              double (&x)[6], float (&dv)[3]) {
    const double h = tn - q.t[u];
    const float hf = (float)h;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int64_t k = d * q.n + u;
        const float a = q.af[k], j = q.jf[k];
        const float dx = hf * hf * (0.5f * a + hf * (j * (1.0f / 6.0f)));
        dv[d] = hf * (a + hf * (0.5f * j));
        const double v = q.vel[k];
        x[d] = fma(h, v, q.pos[k]) + (double)dx;
        x[3 + d] = v;  // the velocity change dv is added in FP32 to the packed offset
    }
}

constexpr int kPackMaxPer = 4;  // slots per thread in block_pack_kernel (tc <= 4 NT)

// FP64 is scarce on this part (about 1/64 of the FP32 rate), so the tile
// centre never needs an FP64 reduction.  After a re-sort (FRESH) it is the
// mean of the FP32-rounded predicted positions (velocities); otherwise the
// tile holds the same particles as at the previous pack, and the centre is
// that pack's centre moved by the mean of its FP32 offsets (their mean
// position then) -- FP32 data only.  Any centre near the tile serves: offsets
// are FP64 differences from it, rounded once to FP32.  It is stored as a
// float (lo = 0).  One CTA per tile, so the previous offsets are all read
// before the CTA overwrites them.
template <int NT, bool FRESH>
__global__ void __launch_bounds__(NT) block_pack_kernel(const BlockPackParams q) {
    __shared__ float redf[NT / 32][8];
    __shared__ double cen[6];
    __shared__ bool last;
    __shared__ int total;
    const int tile = blockIdx.x;
    // this step's time from the previous step's state (every CTA reads it
    // before the last one, below, stores it)
    const long long tnq = block_next_time_q(q.sc->t_next_q, q.sc->n_active, q.sc->level, q.dt_max, q.dt_min);
    const double tn = (double)tnq * q.dt_min;
    const bool live = tn <= q.sc->t_end;
    const ClusterDev cl = q.cl[q.tile_cluster[tile]];
    const int base = tile * q.tc;
    const int per = q.tc / NT;
    float sf[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // position, velocity sums (6), count, active count
    double x[kPackMaxPer][6];
    float dvel[kPackMaxPer][3];
    bool act[kPackMaxPer];
#pragma unroll
    for (int r = 0; r < kPackMaxPer; ++r) {
        act[r] = false;
        const int slot = base + threadIdx.x + NT * r;
        if (r < per && slot - cl.slot_begin < cl.n) {
            const int64_t u = q.perm[slot];
            predict_mixed(q, u, tn, x[r], dvel[r]);
            if (FRESH) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    sf[d] += (float)x[r][d];
                    sf[3 + d] += (float)x[r][3 + d] + dvel[r][d];
                }
            } else {
                sf[0] += q.px[slot];
                sf[1] += q.py[slot];
                sf[2] += q.pz[slot];
                sf[3] += q.pvx[slot];
                sf[4] += q.pvy[slot];
                sf[5] += q.pvz[slot];
            }
            sf[6] += 1.0f;
            act[r] = live && q.tq[u] == tnq;
            sf[7] += act[r] ? 1.0f : 0.0f;
        }
    }
    // CTA sum in FP32, fixed order (counts are exact: at most tc)
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sf[k] += __shfl_xor_sync(0xffffffffu, sf[k], o);
    if (threadIdx.x % 32 == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) redf[threadIdx.x / 32][k] = sf[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float v = redf[0][k];
            for (int w = 1; w < NT / 32; ++w) v += redf[w][k];
            sf[k] = v;
        }
        const float inv = sf[6] > 0.0f ? 1.0f / sf[6] : 0.0f;
        float h[6];
        if (!FRESH) {
            const float4 p0 = q.chl[2 * tile], v0 = q.vchl[2 * tile];
            const float prev[6] = {p0.x, p0.y, p0.z, v0.x, v0.y, v0.z};
#pragma unroll
            for (int d = 0; d < 6; ++d) h[d] = prev[d] + sf[d] * inv;
        } else {
#pragma unroll
            for (int d = 0; d < 6; ++d) h[d] = sf[d] * inv;
        }
#pragma unroll
        for (int d = 0; d < 6; ++d) cen[d] = (double)h[d];
        q.chl[2 * tile + 0] = make_float4(h[0], h[1], h[2], 0.0f);
        q.chl[2 * tile + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        q.vchl[2 * tile + 0] = make_float4(h[3], h[4], h[5], 0.0f);
        q.vchl[2 * tile + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        q.tile_cnt[tile] = (int)sf[7];
    }
    __syncthreads();
    double c[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) c[d] = cen[d];
#pragma unroll
    for (int r = 0; r < kPackMaxPer; ++r) {
        const int slot = base + threadIdx.x + NT * r;
        if (r >= per) break;
        if (slot - cl.slot_begin < cl.n) {
            q.px[slot] = (float)(x[r][0] - c[0]);
            q.py[slot] = (float)(x[r][1] - c[1]);
            q.pz[slot] = (float)(x[r][2] - c[2]);
            if (FRESH) q.pm[slot] = (float)q.mass[q.perm[slot]];  // else unchanged
            // velocity offsets: FP64 difference from the centre, then the FP32
            // change (two roundings, well inside the jerk's tolerance)
            q.pvx[slot] = (float)(x[r][3] - c[3]) + dvel[r][0];
            q.pvy[slot] = (float)(x[r][4] - c[4]) + dvel[r][1];
            q.pvz[slot] = (float)(x[r][5] - c[5]) + dvel[r][2];
            q.flag[slot] = act[r];
        } else {
            q.px[slot] = kPadOffset;
            q.py[slot] = kPadOffset;
            q.pz[slot] = kPadOffset;
            q.pm[slot] = 0.0f;
            q.pvx[slot] = q.pvy[slot] = q.pvz[slot] = 0.0f;
            q.flag[slot] = 0;
        }
    }
    // the last CTA reads only the tile counts (thread 0's writes); the packed
    // data is for later kernels
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&q.sc->ticket_pack, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    block_exclusive_scan<NT>(q.tile_cnt, q.tile_off, q.n_tiles, &total);
    __syncthreads();
    if (threadIdx.x == 0) {
        q.sc->t_next_q = tnq;
        q.sc->t_next = tn;
        plan_step(q.tile_off, total, q.n_tiles, q.tile_first, q.ncl, q.cl, q.cs, q.workers, q.max_split,
                  q.act_begin, q.act_n, q.ich_off, q.item_off, q.sc, q.queue_head, q.few_max, q.cs_large,
                  q.workers_large, q.large_min, q.partial_cap);
        q.sc->ticket_pack = 0;
    }
}

// Work item k -> (cluster, i-chunk of the active list, j-range split).
__device__ __forceinline__ SubItem make_item(int k, int ncl, const ClusterDev *__restrict__ cl, int cs,
                                             int split, const int *__restrict__ act_begin,
                                             const int *__restrict__ act_n,
                                             const int *__restrict__ ich_off,
                                             const int *__restrict__ item_off) {
    int lo = 0, hi = ncl;  // cluster c with item_off[c] <= k < item_off[c + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (item_off[mid] <= k) lo = mid;
        else hi = mid;
    }
    const int c = lo;
    const ClusterDev d = cl[c];
    const int sc_c = split < d.n_jt ? split : (d.n_jt > 0 ? d.n_jt : 1);
    const int local = k - item_off[c];
    const int ch = local / sc_c, s = local % sc_c;
    SubItem it;
    it.a0 = act_begin[c] + ch * cs;
    it.na = min(cs, act_n[c] - ch * cs);
    it.cluster = c;
    it.chunk = ich_off[c] + ch;
    it.jt0 = (int)((int64_t)s * d.n_jt / sc_c);
    it.jt1 = (int)((int64_t)(s + 1) * d.n_jt / sc_c);
    it.split = s;
    it.nsplit = sc_c;
    it.pbase = sc_c > 1 ? it.chunk * split : 0;
    it.pad = 0;
    return it;
}

// Ordered compaction of one run of flags [begin, end): the k-th set flag in
// order writes its index to act[off + k] (warp ballots, warps in order).
template <int NT>
__device__ __forceinline__ void compact_run(const uint8_t *__restrict__ flag, int64_t begin, int64_t end,
                                            int off, int32_t *__restrict__ act) {
    __shared__ int warp_cnt[NT / 32];
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    for (int64_t b = begin; b < end; b += NT) {
        const int64_t i = b + threadIdx.x;
        const int f = i < end ? flag[i] : 0;
        const unsigned mask = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_cnt[w] = __popc(mask);
        __syncthreads();
        int o = off;
        for (int k = 0; k < w; ++k) o += warp_cnt[k];
        if (f) act[o + __popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
        for (int k = 0; k < NT / 32; ++k) off += warp_cnt[k];
        __syncthreads();
    }
}

// Compaction stage 3 (FP64 path): ordered scatter of the active rows to act[]
// in row order within each cluster.
__global__ void block_scatter_kernel(const uint8_t *__restrict__ flag, const Chunk *__restrict__ chunks,
                                     const int *__restrict__ chunk_off, int32_t *__restrict__ act) {
    const Chunk ch = chunks[blockIdx.x];
    const int off = __ldcg(chunk_off + blockIdx.x);
    compact_run<256>(flag, ch.begin, ch.end, off, act);
}

// Work queue (FP64 path).
__global__ void block_items_kernel(int ncl, const ClusterDev *__restrict__ cl,
                                   const int *__restrict__ act_begin, const int *__restrict__ act_n,
                                   const int *__restrict__ ich_off, const int *__restrict__ item_off,
                                   const BlockScalars *__restrict__ sc, int max_items,
                                   SubItem *__restrict__ items, SubItem *__restrict__ info) {
    const int n_items = sc->n_items;
    const int split = sc->split;
    const int cs = sc->cs;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_items && k < max_items;
         k += gridDim.x * blockDim.x) {
        const SubItem it = make_item(k, ncl, cl, cs, split, act_begin, act_n, ich_off, item_off);
        items[k] = it;
        if (it.split == 0) info[it.chunk] = it;
    }
}

// F32C queue: one CTA per centre tile compacts the tile's active slots to
// act[] (slot order within each cluster), and all threads build the items.
template <int NT>
__global__ void __launch_bounds__(NT)
    block_queue_kernel(const uint8_t *__restrict__ flag, int tc, const int *__restrict__ tile_cnt,
                       const int *__restrict__ tile_off, int32_t *__restrict__ act, int ncl,
                       const ClusterDev *__restrict__ cl, const int *__restrict__ act_begin,
                       const int *__restrict__ act_n, const int *__restrict__ ich_off,
                       const int *__restrict__ item_off, const BlockScalars *__restrict__ sc,
                       int max_items, SubItem *__restrict__ items, SubItem *__restrict__ info) {
    const int tile = blockIdx.x;
    if (tile_cnt[tile] > 0)  // uniform over the CTA
        compact_run<NT>(flag, (int64_t)tile * tc, (int64_t)(tile + 1) * tc, __ldcg(tile_off + tile), act);
    const int n_items = sc->n_items;
    const int split = sc->split;
    const int cs = sc->cs;
    for (int k = blockIdx.x * NT + threadIdx.x; k < n_items && k < max_items; k += gridDim.x * NT) {
        const SubItem it = make_item(k, ncl, cl, cs, split, act_begin, act_n, ich_off, item_off);
        items[k] = it;
        if (it.split == 0) info[it.chunk] = it;
    }
}

// The corrector as a pass over the active list: row = act[k] (FP64 path).
__global__ void block_correct_kernel(const BlockCorrect c, const int32_t *__restrict__ act,
                                     const double *__restrict__ a1, const double *__restrict__ j1,
                                     const double *__restrict__ p1) {
    const double tn = c.sc->t_next;
    const long long tnq = c.sc->t_next_q;
    const int n_active = c.sc->n_active;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_active; k += gridDim.x * blockDim.x) {
        const int64_t i = act[k];
        double A1[3], J1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            A1[d] = a1[d * c.n + i];
            J1[d] = j1[d * c.n + i];
        }
        correct_particle(c, i, A1, J1, p1[i], tn, tnq);
    }
}

int grid_of(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
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
                               const int32_t *act, BlockScalars *sc, double *few_part, const SubItem *info,
                               cudaStream_t s) {
    const int64_t units = (int64_t)max_chunks * ((max_cs + 31) / 32);
    const int grid = (int)std::max<int64_t>(kFewCtas, std::min<int64_t>(units, max_ctas));
    subset_tail_kernel<<<grid, kFewThreads, 0, s>>>(prm, act, sc, few_part, info);
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

cudaError_t launch_block_init(int64_t n, const double *acc, const double *jerk, double dt_max,
                              double dt_min, double eta_s, double *t, double *dt, long long *tq,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    block_init_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, acc, jerk, dt_max, dt_min, eta_s, t, dt, tq);
    return cudaGetLastError();
}

cudaError_t launch_block_shadow(int64_t n, const double *acc, const double *jerk, float *af, float *jf,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    block_shadow_kernel<<<grid_of(3 * n, 256), 256, 0, s>>>(3 * n, acc, jerk, af, jf);
    return cudaGetLastError();
}

cudaError_t launch_block_levels(int64_t n, const double *dt, double dt_max, double dt_min,
                                const Chunk *chunks, int n_chunks, const long long *tq, double *part,
                                BlockScalars *sc, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    block_levels_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, dt, dt_max, sc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    block_min_kernel<<<n_chunks, kMinThreads, 0, s>>>(tq, chunks, reinterpret_cast<long long *>(part),
                                                      n_chunks, dt_min, sc);
    return cudaGetLastError();
}

cudaError_t launch_block_prepare(const BlockLaunch &b, cudaStream_t s, int *kernels) {
    cudaError_t e;
#define NB_BL(x)                        \
    do {                                \
        x;                              \
        e = cudaGetLastError();         \
        if (e != cudaSuccess) return e; \
        ++*kernels;                     \
    } while (0)
    if (!b.px)  // the F32C path has t_next from the previous step's last kernel
        NB_BL((block_min_kernel<<<b.n_chunks, kMinThreads, 0, s>>>(
            b.tq, b.chunks, reinterpret_cast<long long *>(b.part), b.n_chunks, b.dt_min, b.sc)));
    if (b.px) {
        if (b.tc <= 0 || b.tc % 128 != 0 || b.tc > kPackMaxPer * (b.tc % 256 == 0 ? 256 : 128))
            return cudaErrorInvalidValue;
        BlockPackParams q{};
        q.perm = b.perm; q.cl = b.cl; q.tile_cluster = b.tile_cluster; q.tc = b.tc;
        q.n_tiles = b.n_tiles; q.n = b.n; q.mass = b.mass; q.t = b.t; q.tq = b.tq; q.af = b.af; q.jf = b.jf;
        q.pos = b.pos; q.vel = b.vel;
        q.px = b.px; q.py = b.py; q.pz = b.pz; q.pm = b.pm;
        q.pvx = b.pvx; q.pvy = b.pvy; q.pvz = b.pvz; q.chl = b.chl; q.vchl = b.vchl;
        q.flag = b.flag; q.tile_cnt = b.cnt; q.tile_off = b.chunk_off; q.tile_first = b.tile_first;
        q.ncl = b.ncl; q.cs = b.cs; q.workers = b.workers; q.max_split = b.max_split;
        q.act_begin = b.act_begin; q.act_n = b.act_n; q.ich_off = b.ich_off; q.item_off = b.item_off;
        q.sc = b.sc; q.queue_head = b.queue_head; q.few_max = b.few_max;
        q.cs_large = b.cs_large; q.workers_large = b.workers_large; q.large_min = b.large_min;
        q.partial_cap = b.partial_cap;
        q.dt_max = b.dt_max;
        q.dt_min = b.dt_min;
        if (b.tc % 256 == 0) {
            if (b.fresh) NB_BL((block_pack_kernel<256, true><<<b.n_tiles, 256, 0, s>>>(q)));
            else NB_BL((block_pack_kernel<256, false><<<b.n_tiles, 256, 0, s>>>(q)));
        } else {
            if (b.fresh) NB_BL((block_pack_kernel<128, true><<<b.n_tiles, 128, 0, s>>>(q)));
            else NB_BL((block_pack_kernel<128, false><<<b.n_tiles, 128, 0, s>>>(q)));
        }
    } else {
        NB_BL((block_predict_kernel<<<grid_of(b.n, 256), 256, 0, s>>>(
            b.n, b.sc, b.t, b.tq, b.pos, b.vel, b.acc, b.jerk, b.xp, b.vp, b.flag)));
        NB_BL((block_count_kernel<<<b.n_chunks, 256, 0, s>>>(b.flag, b.chunks, b.cnt)));
        NB_BL((block_plan_kernel<<<1, kScan, 0, s>>>(b.cnt, b.n_chunks, b.chunk_first, b.ncl, b.cl, b.cs,
                                                      b.workers, b.max_split, b.chunk_off, b.act_begin,
                                                      b.act_n, b.ich_off, b.item_off, b.sc)));
    }
    return cudaSuccess;
}

cudaError_t launch_block_queue(const BlockLaunch &b, cudaStream_t s, int *kernels) {
    cudaError_t e;
    if (b.px) {
        if (b.tc % 256 == 0)
            NB_BL((block_queue_kernel<256><<<b.n_tiles, 256, 0, s>>>(
                b.flag, b.tc, b.cnt, b.chunk_off, b.act, b.ncl, b.cl, b.act_begin, b.act_n, b.ich_off,
                b.item_off, b.sc, b.max_items, b.items, b.info)));
        else
            NB_BL((block_queue_kernel<128><<<b.n_tiles, 128, 0, s>>>(
                b.flag, b.tc, b.cnt, b.chunk_off, b.act, b.ncl, b.cl, b.act_begin, b.act_n, b.ich_off,
                b.item_off, b.sc, b.max_items, b.items, b.info)));
    } else {
        NB_BL((block_scatter_kernel<<<b.n_chunks, 256, 0, s>>>(b.flag, b.chunks, b.chunk_off, b.act)));
        NB_BL((block_items_kernel<<<grid_of(b.max_items, 256), 256, 0, s>>>(
            b.ncl, b.cl, b.act_begin, b.act_n, b.ich_off, b.item_off, b.sc, b.max_items, b.items,
            b.info)));
    }
    return cudaSuccess;
}
#undef NB_BL


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

cudaError_t launch_block_correct(const BlockCorrect &c, const int32_t *act, const double *a1,
                                 const double *j1, const double *p1, cudaStream_t s) {
    if (c.n <= 0) return cudaSuccess;
    // grid-stride over the active list: a few waves suffice for every particle
    const int grid = std::min(grid_of(c.n, 256), 2 * 152);
    block_correct_kernel<<<grid, 256, 0, s>>>(c, act, a1, j1, p1);
    return cudaGetLastError();
}

}  // namespace nbody
