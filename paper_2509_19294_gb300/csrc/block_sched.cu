// block_sched.cu -- individual (block) time steps: the device-side schedule
// (times, prediction and packing, plan, compaction, corrector pass).
//
// Around the Hermite scheme each particle keeps its own time t_i and a
// power-of-two step dt_i (Makino & Aarseth 1992; the paper computes the jerk,
// Sec. 3, but does not describe its stepping).  One block step, all on the
// device so that it is a fixed kernel sequence a CUDA graph can replay
// (F32C; the FP64 path keeps separate predict / count / plan / scatter /
// items / correct kernels around its own subset kernel):
//   1. the step's time t_next = min_i (t_i + dt_i): the next multiple of the
//      smallest occupied step (per-level counts kept by the corrector), taken
//      by every CTA of block_pack_kernel (block_min_kernel, an integer min in
//      units of dt_min, runs at the start and on the FP64 path)
//   2. block_pack_kernel: predict every particle to t_next in FP32 from the
//      slot-ordered mirror (offsets from per-tile frames moving at constant
//      velocity), pack it as the j-set (the jerk path's geometry) with the
//      low parts of the position offsets, flag and count the active slots per
//      tile; the last CTA plans the step (offsets, regime, and the force
//      pass's work: the (i-chunk, j-tile) units cut into one even range per
//      CTA).  block_fresh_kernel replaces it after a re-sort and at the start
//      of an advance: it predicts from the FP64 rows, sets the frames and
//      writes the mirror.
//   3. block_compact_kernel: ordered compaction of the active slots
//   4. the force pass (block_force.cu): the small-set and the large-set subset
//      kernels, then subset_tail_kernel, which either runs the few-particle
//      pass (<= kFewMax active; the subset kernels then have no work) or sums
//      the partials of the i-chunks that several CTAs' ranges share, in order
//   5. the Hermite corrector and next-step choice, in the epilogue of 4
#include <algorithm>
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "block_common.cuh"
#include "nbody_internal.h"

namespace nbody {

namespace {

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
                  act_n, ich_off, item_off, sc, 0, 0, 0, 0, 0);
}

// F32C: one CTA per centre tile of the j-set.  Predicts the tile's particles to
// t_next, packs them as the j-set (FP32 offsets from the tile centre, FP32
// masses, pads far away with mass 0), flags the active slots and counts them.
// The last CTA to finish (ticket) scans the tile counts and plans the step.
// Two forms: block_fresh_kernel (after a re-sort, at the start of an advance)
// gathers the FP64 rows through perm, sets each tile's frame and writes the
// slot mirror; block_pack_kernel (every other step) reads only the FP32 mirror.
struct BlockPackParams {
    const int32_t *perm;
    const ClusterDev *cl;
    const int32_t *tile_cluster;
    int tc, n_tiles;
    int64_t n;
    const double *mass, *t, *pos, *vel, *acc, *jerk;  // rows (fresh pack)
    const long long *tq;                               // rows (fresh pack)
    SlotMirror m;
    float *px, *py, *pz, *pm, *pvx, *pvy, *pvz;
    float *pxl, *pyl, *pzl;  // low parts: px + pxl is the offset to ~2^-48 relative
    float4 *chl, *vchl;
    uint8_t *flag;  // per slot
    int *tile_cnt, *tile_off;
    const int32_t *tile_first;
    int ncl, cs, workers, max_split;
    int *act_begin, *act_n, *ich_off, *item_off;
    long long *work_off;  // per cluster: first (i-chunk, j-tile) unit of the step's work
    BlockScalars *sc;
    int few_max;
    int cs_large, workers_large, large_min;
    long long partial_cap;  // doubles in the split-partial buffer
    int sms;
    unsigned long long *trace;  // per-step trace ring (2 values a record) or null
    int trace_cap;
    double dt_max, dt_min;
    float dt_min_f;  // dt_min as a float (exact: a power of two >= 2^-126)
};

// Per-step trace (NBODY_FLAG_TRACE): as the step starts, the global timer and
// the previous step's active count at record `blocks` (the steps planned so
// far).  A pack after a step that moved nobody (the batch's steps past t_end)
// leaves the record alone, so that the last real step's end stays; a fresh
// pack (the start of an advance call, a re-sort) always writes, so that a
// call's first step starts at its own record.
__device__ __forceinline__ void trace_step(const BlockPackParams &q, bool always) {
    if (!q.trace || blockIdx.x != 0 || threadIdx.x != 0) return;
    const int moved = q.sc->n_active;
    if (!always && moved == 0) return;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    unsigned long long *r = q.trace + 2 * (q.sc->blocks % q.trace_cap);
    r[0] = t;
    r[1] = (unsigned long long)moved;
}

// The end record of an advance call's last step when no pack followed it in
// the call (the record that pack would have written).
__global__ void block_trace_end_kernel(const BlockScalars *__restrict__ sc, unsigned long long *trace, int cap) {
    const int moved = sc->n_active;
    if (moved == 0) return;  // a pack after the last step wrote it
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    unsigned long long *r = trace + 2 * (sc->blocks % cap);
    r[0] = t;
    r[1] = (unsigned long long)moved;
}

// The step's time in units of dt_min (block_next_time_q with the level scan
// done by one warp-wide ballot instead of a loop of dependent loads; every
// lane of the warp calls it).
__device__ __forceinline__ long long next_time_q_warp(const BlockScalars *sc, double dt_max, double dt_min) {
    const int lane = threadIdx.x % 32;
    const long long tq_now = sc->t_next_q;
    const int n_moved = sc->n_active;
    const unsigned lo = __ballot_sync(0xffffffffu, sc->level[lane] != 0);
    const unsigned hi = __ballot_sync(0xffffffffu, sc->level[lane + 32] != 0);
    if (n_moved == 0) return tq_now;
    const int kmax = block_level(dt_min, dt_max);
    unsigned long long occ = ((unsigned long long)hi << 32) | lo;
    if (kmax < 63) occ &= (2ULL << kmax) - 1;  // levels 0 .. kmax
    const int k = occ ? 63 - __clzll((long long)occ) : 0;
    const int sh = kmax - k;  // the smallest occupied step is 2^sh dt_min
    return ((tq_now >> sh) + 1) << sh;
}

// The last CTA to arrive scans the tile counts and plans the step.
template <int NT>
__device__ __forceinline__ void pack_tail(const BlockPackParams &q, long long tnq, bool fresh) {
    __shared__ bool last;
    __shared__ int total;
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
        q.sc->t_next = (double)tnq * q.dt_min;
        if (fresh) q.sc->frame_t0q = tnq;
        plan_step(q.tile_off, total, q.n_tiles, q.tile_first, q.ncl, q.cl, q.cs, q.workers, q.max_split,
                  q.act_begin, q.act_n, q.ich_off, q.item_off, q.sc, q.few_max, q.cs_large,
                  q.workers_large, q.large_min, q.partial_cap, q.work_off, q.sms);
        q.sc->ticket_pack = 0;
    }
}

// Hermite predictor from the rows (fresh pack): x + h v in FP64, the
// higher-order terms h^2 (a/2 + h a'/6) and h (a + h a'/2) in FP32 (small
// against the step's displacement; their FP32 rounding stays far below that of
// the packed FP32 offsets).  The velocity change is returned apart, for the
// packed offset.
__device__ __forceinline__ void predict_rows(const BlockPackParams &q, int64_t u, double tn, double (&x)[6],
                                             float (&dv)[3]) {
    const double h = tn - q.t[u];
    const float hf = (float)h;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int64_t k = d * q.n + u;
        const float a = (float)q.acc[k], j = (float)q.jerk[k];
        const float dx = hf * hf * (0.5f * a + hf * (j * (1.0f / 6.0f)));
        dv[d] = hf * (a + hf * (0.5f * j));
        const double v = q.vel[k];
        x[d] = fma(h, v, q.pos[k]) + (double)dx;
        x[3 + d] = v;  // the velocity change dv is added in FP32 to the packed offset
    }
}

// Fresh pack: the tile's frame is set at t0 = t_next to the FP32 mean of its
// particles' predicted positions and velocities (no FP64 reduction: any centre
// near the tile serves, offsets are FP64 differences rounded once to FP32);
// the mirror takes each particle's offsets from the frame at its own time.
template <int NT, int PER>
__global__ void __launch_bounds__(NT) block_fresh_kernel(const BlockPackParams q) {
    trace_step(q, true);
    __shared__ float redf[NT / 32][8];
    __shared__ float cen[6];
    const int tile = blockIdx.x;
    // this step's time from the previous step's state (every CTA reads it
    // before the last one, in pack_tail, stores it)
    const long long tnq = next_time_q_warp(q.sc, q.dt_max, q.dt_min);
    const double tn = (double)tnq * q.dt_min;
    const bool live = tn <= q.sc->t_end;
    const ClusterDev cl = q.cl[q.tile_cluster[tile]];
    const int base = tile * NT * PER;  // tc = NT * PER slots per tile
    float sf[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // position, velocity sums (6), count, active count
    double x[PER][6];
    float dvel[PER][3];
    bool act[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        act[r] = false;
        const int slot = base + threadIdx.x + NT * r;
        if (slot - cl.slot_begin < cl.n) {
            const int64_t u = q.perm[slot];
            predict_rows(q, u, tn, x[r], dvel[r]);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                sf[d] += (float)x[r][d];
                sf[3 + d] += (float)x[r][3 + d] + dvel[r][d];
            }
            sf[6] += 1.0f;
            act[r] = live && q.tq[u] == tnq;
            sf[7] += act[r] ? 1.0f : 0.0f;
        }
    }
    // CTA sums in FP32, fixed order (counts are exact: at most tc)
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
#pragma unroll
        for (int d = 0; d < 6; ++d) cen[d] = sf[d] * inv;
        q.chl[2 * tile + 0] = make_float4(cen[0], cen[1], cen[2], 0.0f);
        q.chl[2 * tile + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // c(t0) = c0 exactly
        q.vchl[2 * tile + 0] = make_float4(cen[3], cen[4], cen[5], 0.0f);
        q.vchl[2 * tile + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int d = 0; d < 3; ++d) q.m.c0[(int64_t)d * q.n_tiles + tile] = (double)cen[d];
        q.tile_cnt[tile] = (int)sf[7];
    }
    __syncthreads();
    double c[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) c[d] = (double)cen[d];
    const double inv_dt_min = recip_pow2(q.dt_min);
    const int64_t np = q.m.n_pad;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int slot = base + threadIdx.x + NT * r;
        if (slot - cl.slot_begin < cl.n) {
            const int64_t u = q.perm[slot];
            {
                float hi[3], lo[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const double o = x[r][d] - c[d];
                    hi[d] = (float)o;
                    lo[d] = (float)(o - (double)hi[d]);
                }
                q.px[slot] = hi[0];
                q.py[slot] = hi[1];
                q.pz[slot] = hi[2];
                q.pxl[slot] = lo[0];
                q.pyl[slot] = lo[1];
                q.pzl[slot] = lo[2];
            }
            q.pm[slot] = (float)q.mass[u];
            // velocity offsets: FP64 difference from the centre, then the FP32
            // change (two roundings, well inside the jerk's tolerance)
            q.pvx[slot] = (float)(x[r][3] - c[3]) + dvel[r][0];
            q.pvy[slot] = (float)(x[r][4] - c[4]) + dvel[r][1];
            q.pvz[slot] = (float)(x[r][5] - c[5]) + dvel[r][2];
            q.flag[slot] = act[r];
            // the mirror: offsets from the frame at the particle's own time t_i
            const double ti = q.t[u], back = ti - tn;  // <= 0, exact (multiples of dt_min)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int64_t k = d * q.n + u, ks = d * np + slot;
                const double xr = q.pos[k] - fma(c[3 + d], back, c[d]);
                const float hi = (float)xr;
                q.m.xr[ks] = hi;
                q.m.xl[ks] = (float)(xr - (double)hi);
                q.m.vr[ks] = (float)(x[r][3 + d] - c[3 + d]);
                q.m.af[ks] = (float)q.acc[k];
                q.m.jf[ks] = (float)q.jerk[k];
            }
            q.m.tcq[slot] = (long long)(ti * inv_dt_min);
            q.m.tq[slot] = q.tq[u];
        } else {
            q.px[slot] = kPadOffset;
            q.py[slot] = kPadOffset;
            q.pz[slot] = kPadOffset;
            q.pxl[slot] = q.pyl[slot] = q.pzl[slot] = 0.0f;
            q.pm[slot] = 0.0f;
            q.pvx[slot] = q.pvy[slot] = q.pvz[slot] = 0.0f;
            q.flag[slot] = 0;
        }
    }
    pack_tail<NT>(q, tnq, true);
}

// Every other step: FP32 only.  With k = t_next - t_i (units of dt_min, exact
// h = k dt_min), the offset from the frame at t_next is
// xr + (xl + h (vr + h (a/2 + h a'/6))), rounded to FP32 once against the
// pair's high part, and the velocity offset vr + h (a + h a'/2);
// the tile's centre is the frame at t_next, c0 + cv (t_next - t0), evaluated
// in FP64 once per tile and stored as a float pair.  Pads keep what the fresh
// pack wrote.
template <int NT, int PER>
__global__ void __launch_bounds__(NT) block_pack_kernel(const BlockPackParams q) {
    trace_step(q, false);
    __shared__ int wcnt[NT / 32];
    const int tile = blockIdx.x;
    const long long tnq = next_time_q_warp(q.sc, q.dt_max, q.dt_min);
    const bool live = tnq <= q.sc->t_end_q;
    double c0[3] = {0.0, 0.0, 0.0};
    float4 cv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    long long t0q = 0;
    if (threadIdx.x == 0) {  // the frame (loads issued early)
#pragma unroll
        for (int d = 0; d < 3; ++d) c0[d] = q.m.c0[(int64_t)d * q.n_tiles + tile];
        cv = q.vchl[2 * tile];
        t0q = q.sc->frame_t0q;
    }
    const ClusterDev cl = q.cl[q.tile_cluster[tile]];
    const int base = tile * NT * PER;
    const int64_t np = q.m.n_pad;
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int slot = base + threadIdx.x + NT * r;
        if (slot - cl.slot_begin < cl.n) {
            // h = k dt_min, 0 <= k <= dt_max / dt_min <= 2^40: two exact 32-bit
            // conversions and one rounding (no 64-bit conversion, which runs
            // on the FP64 pipe)
            const long long k = tnq - q.m.tcq[slot];
            const float kf = fmaf((float)(int)(k >> 24), 16777216.0f, (float)(int)(k & 0xFFFFFF));
            const float hf = kf * q.dt_min_f;
            float o[6], ol[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int64_t ks = d * np + slot;
                const float xr = q.m.xr[ks], xl = q.m.xl[ks], vr = q.m.vr[ks], a = q.m.af[ks], j = q.m.jf[ks];
                const float t = xl + hf * (vr + hf * (0.5f * a + hf * (j * (1.0f / 6.0f))));
                // o + ol = xr + t exactly (TwoSum)
                const float sum = __fadd_rn(xr, t), bb = __fsub_rn(sum, xr);
                o[d] = sum;
                ol[d] = __fadd_rn(__fsub_rn(xr, __fsub_rn(sum, bb)), __fsub_rn(t, bb));
                o[3 + d] = vr + hf * (a + hf * (0.5f * j));
            }
            q.px[slot] = o[0];
            q.py[slot] = o[1];
            q.pz[slot] = o[2];
            q.pxl[slot] = ol[0];
            q.pyl[slot] = ol[1];
            q.pzl[slot] = ol[2];
            q.pvx[slot] = o[3];
            q.pvy[slot] = o[4];
            q.pvz[slot] = o[5];
            const bool a = live && q.m.tq[slot] == tnq;
            q.flag[slot] = a;
            cnt += a ? 1 : 0;
        }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (threadIdx.x % 32 == 0) wcnt[threadIdx.x / 32] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int total = 0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) total += wcnt[w];
        q.tile_cnt[tile] = total;
        const double dtf = (double)(tnq - t0q) * q.dt_min;
        const float cvd[3] = {cv.x, cv.y, cv.z};
        float hi[3], lo[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double c = fma((double)cvd[d], dtf, c0[d]);
            hi[d] = (float)c;
            lo[d] = (float)(c - (double)hi[d]);
        }
        q.chl[2 * tile + 0] = make_float4(hi[0], hi[1], hi[2], 0.0f);
        q.chl[2 * tile + 1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
    }
    pack_tail<NT>(q, tnq, false);
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

// F32C compaction: one CTA per centre tile writes the tile's active slots to
// act[] (slot order within each cluster); the force pass's work comes from
// the plan (no items).
template <int NT>
__global__ void __launch_bounds__(NT)
    block_compact_kernel(const uint8_t *__restrict__ flag, int tc, const int *__restrict__ tile_cnt,
                       const int *__restrict__ tile_off, int32_t *__restrict__ act) {
    const int tile = blockIdx.x;
    if (tile_cnt[tile] > 0)  // uniform over the CTA
        compact_run<NT>(flag, (int64_t)tile * tc, (int64_t)(tile + 1) * tc, __ldcg(tile_off + tile), act);
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
        correct_particle<false>(c, i, -1, A1, J1, p1[i], tn, tnq);  // no mirror on this path
    }
}

}  // namespace

cudaError_t launch_block_init(int64_t n, const double *acc, const double *jerk, double dt_max,
                              double dt_min, double eta_s, double *t, double *dt, long long *tq,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    block_init_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, acc, jerk, dt_max, dt_min, eta_s, t, dt, tq);
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
        if (b.tc <= 0 || b.tc % 128 != 0 || b.tc > 4 * (b.tc % 256 == 0 ? 256 : 128))  // <= 4 slots a thread
            return cudaErrorInvalidValue;
        BlockPackParams q{};
        q.perm = b.perm; q.cl = b.cl; q.tile_cluster = b.tile_cluster; q.tc = b.tc;
        q.n_tiles = b.n_tiles; q.n = b.n; q.mass = b.mass; q.m = b.mirror;
        q.t = b.t; q.pos = b.pos; q.vel = b.vel; q.acc = b.acc; q.jerk = b.jerk; q.tq = b.tq;
        q.px = b.px; q.py = b.py; q.pz = b.pz; q.pm = b.pm;
        q.pxl = b.pxl; q.pyl = b.pyl; q.pzl = b.pzl;
        q.pvx = b.pvx; q.pvy = b.pvy; q.pvz = b.pvz; q.chl = b.chl; q.vchl = b.vchl;
        q.flag = b.flag; q.tile_cnt = b.cnt; q.tile_off = b.chunk_off; q.tile_first = b.tile_first;
        q.ncl = b.ncl; q.cs = b.cs; q.workers = b.workers; q.max_split = b.max_split;
        q.act_begin = b.act_begin; q.act_n = b.act_n; q.ich_off = b.ich_off; q.item_off = b.item_off;
        q.work_off = b.work_off;
        q.sc = b.sc; q.few_max = b.few_max;
        q.cs_large = b.cs_large; q.workers_large = b.workers_large; q.large_min = b.large_min;
        q.partial_cap = b.partial_cap;
        q.sms = b.sms;
        q.trace = b.trace;
        q.trace_cap = b.trace_cap;
        q.dt_max = b.dt_max;
        q.dt_min = b.dt_min;
        q.dt_min_f = (float)b.dt_min;
        // tc = NT * PER, NT = 256 where tc allows it (checked above: PER <= 4)
#define NB_PACK(NT_, PER_)                                                                  \
    if (b.tc == (NT_) * (PER_)) {                                                           \
        if (b.fresh) NB_BL((block_fresh_kernel<NT_, PER_><<<b.n_tiles, NT_, 0, s>>>(q)));   \
        else NB_BL((block_pack_kernel<NT_, PER_><<<b.n_tiles, NT_, 0, s>>>(q)));            \
        return cudaSuccess;                                                                 \
    }
        NB_PACK(256, 1) NB_PACK(256, 2) NB_PACK(256, 3) NB_PACK(256, 4)
        NB_PACK(128, 1) NB_PACK(128, 3)
#undef NB_PACK
        return cudaErrorInvalidValue;
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
            NB_BL((block_compact_kernel<256><<<b.n_tiles, 256, 0, s>>>(b.flag, b.tc, b.cnt, b.chunk_off,
                                                                     b.act)));
        else
            NB_BL((block_compact_kernel<128><<<b.n_tiles, 128, 0, s>>>(b.flag, b.tc, b.cnt, b.chunk_off,
                                                                     b.act)));
    } else {
        NB_BL((block_scatter_kernel<<<b.n_chunks, 256, 0, s>>>(b.flag, b.chunks, b.chunk_off, b.act)));
        NB_BL((block_items_kernel<<<grid_of(b.max_items, 256), 256, 0, s>>>(
            b.ncl, b.cl, b.act_begin, b.act_n, b.ich_off, b.item_off, b.sc, b.max_items, b.items,
            b.info)));
    }
    return cudaSuccess;
}
#undef NB_BL


cudaError_t launch_block_correct(const BlockCorrect &c, const int32_t *act, const double *a1,
                                 const double *j1, const double *p1, cudaStream_t s) {
    if (c.n <= 0) return cudaSuccess;
    // grid-stride over the active list: a few waves suffice for every particle
    const int grid = std::min(grid_of(c.n, 256), 2 * 152);
    block_correct_kernel<<<grid, 256, 0, s>>>(c, act, a1, j1, p1);
    return cudaGetLastError();
}

cudaError_t launch_block_trace_end(const BlockScalars *sc, unsigned long long *trace, int cap, cudaStream_t s) {
    block_trace_end_kernel<<<1, 1, 0, s>>>(sc, trace, cap);
    return cudaGetLastError();
}

}  // namespace nbody
