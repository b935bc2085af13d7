// block.cu -- individual (block) time steps: forces on the active subset.
//
// Around the Hermite scheme each particle keeps its own time t_i and a
// power-of-two step dt_i (Makino & Aarseth 1992; the paper computes the jerk,
// Sec. 3, but does not describe its stepping).  One block step, all on the
// device so that it is a fixed kernel sequence a CUDA graph can replay:
//   1. t_next = min_i (t_i + dt_i)              (two-stage exact min)
//   2. predict every particle to t_next, flag the active ones
//   3. ordered compaction of the active set per cluster, i-chunk counts,
//      split count and the work queue, built on the device
//   4. pack every predicted particle as the j-set (the jerk path's geometry)
//   5. forces + jerks of the active i-chunks against all j (this file)
//   6. correct the active particles and choose their next steps
// An active particle is evaluated with its own j-set offset and its own tile
// centre: per j-tile each thread forms the exact centre difference for each of
// its particles, so the self pair is exactly zero, as in the full kernels.
#include <algorithm>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "forces_f32c_jerk.cuh"
#include "nbody_internal.h"

namespace nbody {

namespace {

// FP64 epilogue of one active particle: scale by G, remove the self term of
// phi (its own j-tile contributed m_i rsqrt(eps^2) exactly), scatter to its row.
__device__ __forceinline__ void subset_finalize(const F32CJerkParams &p, const ClusterDev &cl,
                                                int slot, const double (&r)[7]) {
    const int64_t u = p.perm[slot];
    double ph = r[6];
    if (cl.eps2f > 0.0f) ph -= (double)__fmul_rn(p.pm[slot], rsqrt_mufu(cl.eps2f));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p.acc[d * p.n + u] = p.G * r[d];
        p.jerk[d * p.n + u] = p.G * r[3 + d];
    }
    if (p.pot) p.pot[u] = -p.G * ph;
}

template <int BLOCK, int P, int TJ, bool EPS_ZERO>
struct SubsetKernel {
    using JK = F32CJerkKernel<BLOCK, P, TJ, EPS_ZERO>;
    static constexpr int NA = JK::NA;
    static constexpr int NC = JK::NC;
    static constexpr int NV = JK::NV;
    static constexpr int NLD = JK::NLD;

    struct Smem {
        float4 j[2][NA][TJ / 4];
        float4 jc[2][4];  // j-tile centre: position hi, lo, velocity hi, lo
        int item;
    };

    __device__ static __forceinline__ void store_tile(Smem &sm, int b, const float4 (&r)[NLD]) {
#pragma unroll
        for (int q = 0; q < NLD; ++q) {
            const int v = threadIdx.x + q * BLOCK;
            if (NV % BLOCK == 0 || v < NV) sm.j[b][v / (TJ / 4)][v % (TJ / 4)] = r[q];
        }
    }

    __device__ static void run(const F32CSubsetParams q) {
        __shared__ Smem sm;
        const F32CJerkParams &p = q.base;
        const int n_items = *q.n_items;
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
                const int pos = threadIdx.x + k * BLOCK;
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
                JK::load_tile(p, gs, reg);
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
                if (more) JK::load_tile(p, gsn, reg);
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
                for (int v = 0; v < TJ / 4; ++v) {
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
            if (it.nsplit <= 1) {
#pragma unroll
                for (int k = 0; k < P; ++k)
                    if (valid[k]) finalize(p, cl, slot[k], res[k]);
                continue;
            }
            // split j-ranges: FP64 partials, summed in a fixed order by
            // subset_reduce_kernel (in parallel over particles and components)
            const int tcs = BLOCK * P;
            double *mine = q.partial + (size_t)(it.pbase + it.split) * NC * tcs;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int l = threadIdx.x + k * BLOCK;
#pragma unroll
                for (int c = 0; c < NC; ++c) mine[c * tcs + l] = res[k][c];
            }
        }
    }

    __device__ static __forceinline__ void finalize(const F32CJerkParams &p, const ClusterDev &cl,
                                                    int slot, const double (&r)[NC]) {
        subset_finalize(p, cl, slot, r);
    }
};

template <int BLOCK, int P, int TJ, int MINB, bool EPS_ZERO>
__global__ void __launch_bounds__(BLOCK, MINB) subset_jerk_kernel(const F32CSubsetParams q) {
    SubsetKernel<BLOCK, P, TJ, EPS_ZERO>::run(q);
}

// Sum the split partials of every chunk and finalise.  Work unit = 32
// particles of one chunk; its 8 warps each sum one contiguous eighth of the
// splits (loads unrolled, so their latencies overlap), then warp 0 adds the
// eight group sums in group order.  The order of every addition is fixed by
// (nsplit, particle), so the result does not depend on scheduling.
constexpr int kReduceWarps = 8;

__global__ void __launch_bounds__(32 * kReduceWarps)
subset_reduce_kernel(const F32CSubsetParams q, const SubItem *__restrict__ info,
                     const BlockScalars *__restrict__ sc, int cs) {
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
            subset_finalize(q.base, q.base.cl[it.cluster], q.act_slot[it.a0 + l], r);
        }
        __syncthreads();
    }
}

struct SubsetShape {
    int block, p, tj, minb;
    bool eps_zero;
    const void *kernel;
};

#define SUBSET(B, P, T, M)                                                                  \
    SubsetShape{B, P, T, M, false, (const void *)subset_jerk_kernel<B, P, T, M, false>},    \
        SubsetShape{B, P, T, M, true, (const void *)subset_jerk_kernel<B, P, T, M, true>}

const SubsetShape kSubsetShapes[] = {SUBSET(64, 2, 256, 4), SUBSET(128, 2, 256, 2),
                                     SUBSET(64, 2, 128, 4), SUBSET(128, 1, 128, 4)};

const SubsetShape *find_subset(int block, int p, int tj, int minb, bool eps_zero) {
    for (const SubsetShape &s : kSubsetShapes)
        if (s.block == block && s.p == p && s.tj == tj && s.minb == minb && s.eps_zero == eps_zero)
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
                                  double dt_min, double eta_s, double *t, double *dt) {
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
    }
}

// Stage 1 of t_next: per chunk, min of t_i + dt_i (exact).
__global__ void block_min_kernel(const double *__restrict__ t, const double *__restrict__ dt,
                                 const Chunk *__restrict__ chunks, double *__restrict__ part) {
    __shared__ double red[8];
    const Chunk ch = chunks[blockIdx.x];
    double m = INFINITY;
    for (int64_t i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) m = fmin(m, t[i] + dt[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) m = fmin(m, red[w]);
        part[blockIdx.x] = m;
    }
}

// Stage 2 of t_next (one CTA): min over the chunk minima.
__global__ void block_tnext_kernel(const double *__restrict__ part, int n_chunks, BlockScalars *sc) {
    __shared__ double red[8];
    double m = INFINITY;
    for (int k = threadIdx.x; k < n_chunks; k += blockDim.x) m = fmin(m, part[k]);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) m = fmin(m, red[w]);
        sc->t_next = m;
    }
}

// Predict every particle to t_next and flag the active ones.
__global__ void block_predict_kernel(int64_t n, const BlockScalars *__restrict__ sc,
                                     const double *__restrict__ t,
                                     const double *__restrict__ dt, const double *__restrict__ pos,
                                     const double *__restrict__ vel, const double *__restrict__ acc,
                                     const double *__restrict__ jerk, double *xp, double *vp,
                                     uint8_t *flag) {
    const double tn = sc->t_next;
    const bool live = tn <= sc->t_end;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double h = tn - t[i], h2 = h * h, h3 = h2 * h;
        for (int d = 0; d < 3; ++d) {
            const int64_t qd = d * n + i;
            xp[qd] = pos[qd] + vel[qd] * h + acc[qd] * h2 / 2.0 + jerk[qd] * h3 / 6.0;
            vp[qd] = vel[qd] + acc[qd] * h + jerk[qd] * h2 / 2.0;
        }
        flag[i] = live && (t[i] + dt[i] == tn);
    }
}

// Compaction stage 1: active count per chunk.
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

// Block-wide exclusive scan of int values (one CTA of kScan threads).
__device__ void block_exclusive_scan(const int *in, int *out, int n, int *total) {
    __shared__ int warp_sums[kScan / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kScan) {
        const int i = base + threadIdx.x;
        const int v = i < n ? in[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x % 32) >= o) x += y;
        }
        if (threadIdx.x % 32 == 31) warp_sums[threadIdx.x / 32] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int w = warp_sums[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (threadIdx.x >= o) w += y;
            }
            warp_sums[threadIdx.x] = w;
        }
        __syncthreads();
        const int warp_off = threadIdx.x >= 32 ? warp_sums[threadIdx.x / 32 - 1] : 0;
        if (i < n) out[i] = carry + warp_off + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[kScan / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Compaction stage 2 (one CTA): chunk offsets, per-cluster active ranges and
// i-chunk counts, the split count and the work-queue size.
__global__ void __launch_bounds__(kScan)
    block_plan_kernel(const int *__restrict__ cnt, int n_chunks, const int32_t *__restrict__ chunk_first,
                      int ncl, const ClusterDev *__restrict__ cl, int cs, int workers, int max_split,
                      int *__restrict__ chunk_off, int *__restrict__ act_begin, int *__restrict__ act_n,
                      int *__restrict__ ich_off, int *__restrict__ item_off, BlockScalars *sc) {
    __shared__ int total;
    block_exclusive_scan(cnt, chunk_off, n_chunks, &total);
    __syncthreads();
    if (threadIdx.x == 0) {
        int chunks = 0;
        for (int c = 0; c < ncl; ++c) {
            const int b = chunk_first[c], e = chunk_first[c + 1];
            const int a0 = b < n_chunks ? chunk_off[b] : total;
            const int a1 = e < n_chunks ? chunk_off[e] : total;
            act_begin[c] = a0;
            act_n[c] = a1 - a0;
            ich_off[c] = chunks;
            chunks += (a1 - a0 + cs - 1) / cs;
        }
        ich_off[ncl] = chunks;
        int split = chunks > 0 ? (2 * workers) / chunks : 1;
        if (split > max_split) split = max_split;
        if (split < 1) split = 1;
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
        if (total > 0) {
            sc->blocks += 1;
            sc->evals += total;
        }
    }
}

// Compaction stage 3: ordered scatter of the active rows (as j-set slots for
// F32C, as rows for F64) to act[] in row order within each cluster.
__global__ void block_scatter_kernel(const uint8_t *__restrict__ flag, const Chunk *__restrict__ chunks,
                                     const int *__restrict__ chunk_off, const int32_t *__restrict__ inv,
                                     int32_t *__restrict__ act) {
    __shared__ int warp_cnt[8];
    __shared__ int base_s;
    const Chunk ch = chunks[blockIdx.x];
    if (threadIdx.x == 0) base_s = chunk_off[blockIdx.x];
    __syncthreads();
    for (int64_t b = ch.begin; b < ch.end; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int f = i < ch.end ? flag[i] : 0;
        const unsigned mask = __ballot_sync(0xffffffffu, f);
        const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
        if (lane == 0) warp_cnt[w] = __popc(mask);
        __syncthreads();
        int off = base_s;
        for (int k = 0; k < w; ++k) off += warp_cnt[k];
        if (f) act[off + __popc(mask & ((1u << lane) - 1u))] = inv ? inv[i] : (int32_t)i;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 0; k < (int)(blockDim.x / 32); ++k) base_s += warp_cnt[k];
        __syncthreads();
    }
}

// Work queue: item k -> (cluster, i-chunk of the active list, j-range split).
__global__ void block_items_kernel(int ncl, const ClusterDev *__restrict__ cl, int cs,
                                   const int *__restrict__ act_begin, const int *__restrict__ act_n,
                                   const int *__restrict__ ich_off, const int *__restrict__ item_off,
                                   const BlockScalars *__restrict__ sc, int max_items,
                                   SubItem *__restrict__ items, SubItem *__restrict__ info) {
    const int n_items = sc->n_items;
    const int split = sc->split;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_items && k < max_items;
         k += gridDim.x * blockDim.x) {
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
        items[k] = it;
        if (s == 0) info[it.chunk] = it;
    }
}

// Inverse of the j-set permutation: inv[row] = slot.
__global__ void inverse_perm_kernel(int64_t n_pad, const int32_t *__restrict__ perm, int32_t *inv) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = perm[s];
        if (u >= 0) inv[u] = (int32_t)s;
    }
}

// Correct the active particles over their own steps and choose the next step.
__global__ void block_correct_kernel(int64_t n, const uint8_t *__restrict__ flag,
                                     const BlockScalars *__restrict__ sc, double *t, double *dt,
                                     double *pos, double *vel, double *acc, double *jerk,
                                     double *pot, const double *__restrict__ a1,
                                     const double *__restrict__ j1, const double *__restrict__ p1,
                                     double dt_max, double dt_min, double eta) {
    const double tn = sc->t_next;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const double h = dt[i], h2 = h * h, h3 = h2 * h;
        double A1[3], J1[3], A2[3], A3[3];
        for (int d = 0; d < 3; ++d) {
            const int64_t q = d * n + i;
            A1[d] = a1[q];
            J1[d] = j1[q];
            const double a0 = acc[q], j0 = jerk[q], v0 = vel[q];
            const double v1 = v0 + (a0 + A1[d]) * h / 2.0 + (j0 - J1[d]) * h2 / 12.0;
            pos[q] = pos[q] + (v0 + v1) * h / 2.0 + (a0 - A1[d]) * h2 / 12.0;
            vel[q] = v1;
            A3[d] = (12.0 * (a0 - A1[d]) + 6.0 * h * (j0 + J1[d])) / h3;
            A2[d] = (-6.0 * (a0 - A1[d]) - h * (4.0 * j0 + 2.0 * J1[d])) / h2 + h * A3[d];
            acc[q] = A1[d];
            jerk[q] = J1[d];
        }
        if (pot) pot[i] = p1[i];
        const double na = sqrt(A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2]);
        const double nj = sqrt(J1[0] * J1[0] + J1[1] * J1[1] + J1[2] * J1[2]);
        const double n2 = sqrt(A2[0] * A2[0] + A2[1] * A2[1] + A2[2] * A2[2]);
        const double n3 = sqrt(A3[0] * A3[0] + A3[1] * A3[1] + A3[2] * A3[2]);
        const double den = nj * n3 + n2 * n2;
        const double da = den > 0.0 ? sqrt(eta * (na * n2 + nj * nj) / den) : dt_max;
        double nd = h;
        while (nd > da && nd > dt_min) nd /= 2.0;
        if (nd == h && da >= 2.0 * h && 2.0 * h <= dt_max && fmod(tn, 2.0 * h) == 0.0) nd = 2.0 * h;
        t[i] = tn;
        dt[i] = nd;
    }
}

int grid_of(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int subset_shapes(int *block, int *p, int *tj, int *minb, int cap) {
    int n = 0;
    for (const SubsetShape &s : kSubsetShapes) {
        if (s.eps_zero) continue;
        if (n < cap) {
            block[n] = s.block;
            p[n] = s.p;
            tj[n] = s.tj;
            minb[n] = s.minb;
        }
        ++n;
    }
    return n;
}

cudaError_t launch_subset_reduce(int max_chunks, int max_ctas, const F32CSubsetParams &prm,
                                 const SubItem *info, const BlockScalars *sc, int cs, cudaStream_t s) {
    const int64_t units = (int64_t)max_chunks * ((cs + 31) / 32);
    if (units <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(units, max_ctas);
    subset_reduce_kernel<<<grid, 32 * kReduceWarps, 0, s>>>(prm, info, sc, cs);
    return cudaGetLastError();
}

int subset_occupancy(int block, int p, int tj, int minb, bool eps_zero) {
    const SubsetShape *s = find_subset(block, p, tj, minb, eps_zero);
    if (!s) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, s->kernel, block, 0) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_block_init(int64_t n, const double *acc, const double *jerk, double dt_max,
                              double dt_min, double eta_s, double *t, double *dt, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    block_init_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, acc, jerk, dt_max, dt_min, eta_s, t, dt);
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
    NB_BL((block_min_kernel<<<b.n_chunks, 256, 0, s>>>(b.t, b.dt, b.chunks, b.part)));
    NB_BL((block_tnext_kernel<<<1, 256, 0, s>>>(b.part, b.n_chunks, b.sc)));
    NB_BL((block_predict_kernel<<<grid_of(b.n, 256), 256, 0, s>>>(
        b.n, b.sc, b.t, b.dt, b.pos, b.vel, b.acc, b.jerk, b.xp, b.vp, b.flag)));
    NB_BL((block_count_kernel<<<b.n_chunks, 256, 0, s>>>(b.flag, b.chunks, b.cnt)));
    NB_BL((block_plan_kernel<<<1, kScan, 0, s>>>(b.cnt, b.n_chunks, b.chunk_first, b.ncl, b.cl, b.cs,
                                                  b.workers, b.max_split, b.chunk_off, b.act_begin,
                                                  b.act_n, b.ich_off, b.item_off, b.sc)));
#undef NB_BL
    return cudaSuccess;
}

cudaError_t launch_block_queue(const BlockLaunch &b, const int32_t *inv, cudaStream_t s, int *kernels) {
    cudaError_t e;
    block_scatter_kernel<<<b.n_chunks, 256, 0, s>>>(b.flag, b.chunks, b.chunk_off, inv, b.act);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    block_items_kernel<<<grid_of(b.max_items, 256), 256, 0, s>>>(
        b.ncl, b.cl, b.cs, b.act_begin, b.act_n, b.ich_off, b.item_off, b.sc, b.max_items, b.items,
        b.info);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *kernels += 2;
    return cudaSuccess;
}

cudaError_t launch_inverse_perm(int64_t n_pad, const int32_t *perm, int32_t *inv, cudaStream_t s) {
    if (n_pad <= 0) return cudaSuccess;
    inverse_perm_kernel<<<grid_of(n_pad, 256), 256, 0, s>>>(n_pad, perm, inv);
    return cudaGetLastError();
}

cudaError_t launch_subset_f32c(int block, int p, int tj, int minb, bool eps_zero, int grid,
                               const F32CSubsetParams &prm, cudaStream_t st) {
    const SubsetShape *sh = find_subset(block, p, tj, minb, eps_zero);
    if (!sh) return cudaErrorNotSupported;
    if (grid <= 0) return cudaSuccess;
    void *args[] = {(void *)&prm};
    return cudaLaunchKernel(sh->kernel, dim3(grid), dim3(block), args, 0, st);
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

cudaError_t launch_block_correct(int64_t n, const uint8_t *flag, const BlockScalars *sc, double *t,
                                 double *dt, double *pos, double *vel, double *acc, double *jerk,
                                 double *pot, const double *a1, const double *j1, const double *p1,
                                 double dt_max, double dt_min, double eta, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    block_correct_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, flag, sc, t, dt, pos, vel, acc, jerk, pot,
                                                         a1, j1, p1, dt_max, dt_min, eta);
    return cudaGetLastError();
}

}  // namespace nbody
