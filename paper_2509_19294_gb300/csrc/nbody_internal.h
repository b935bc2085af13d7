// nbody_internal.h -- shared declarations of the CUDA side of libnbody.so.
//
// Data layout in device memory (F32C mode):
//   * Particles are regrouped into "centre tiles" of Tc = block * p packed slots.
//     Every cluster starts on a tile boundary and is padded up to a multiple of
//     Tc; pad slots carry mass 0 and a far offset so they add exactly nothing.
//   * px/py/pz/pm: float[n_pad] SoA, the FP32 offset of each particle from its
//     tile's centre, and its mass rounded to FP32.
//   * chl: float4[n_tiles][2], each tile's centre as an unevaluated float pair
//     (hi.x + lo.x, ...): the pack kernels store the FP32 mean of the tile's
//     FP32-rounded positions as hi and lo = 0 (offsets are FP64 differences
//     from that centre, rounded once); the block-step pack stores its tile
//     frame's position, an FP64 value, as hi + lo.
//   * perm: int32[n_pad], the caller's row of each packed slot (-1 for pads).
//     Identity within each cluster unless Morton reordering is on.
//   * items: the work queue of the force kernel, one entry per
//     (cluster, i-tile, j-range), largest cost first.
//   * partial: double[slots][4][Tc], FP64 partial sums of the split i-tiles.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace nbody {

constexpr float kPadOffset = 1.0e18f;  // offset of pad slots from their tile centre

struct ClusterDev {
    int64_t user_begin;  // first caller row of the cluster
    int32_t n;           // real particles
    int32_t slot_begin;  // first packed slot (multiple of Tc)
    int32_t n_jt;        // j-tiles of size tj covering the real particles
    float eps2f;         // eps^2 rounded to FP32
    double eps2;         // eps^2 in FP64
};

struct Item {
    int32_t tile;     // global i-tile (centre tile) index
    int32_t cluster;  // owning cluster
    int32_t jt0, jt1; // j-tile range [jt0, jt1), local to the cluster
    int32_t split;    // index of this j-range among the tile's splits
    int32_t nsplit;   // number of splits of this tile (1 = no partials)
    int32_t pbase;    // first partial slot of the tile (when nsplit > 1)
    int32_t pad;
};

// Parameters of the FP32-compensated force kernel (passed by value).
struct F32CParams {
    const float *px, *py, *pz, *pm;
    const float4 *chl;
    const int32_t *perm;
    const ClusterDev *cl;
    const Item *items;
    int32_t n_items;
    int32_t tc;        // centre-tile size (block * p)
    int *counters;     // [0] queue head, [1 + tile] split tickets
    double *partial;   // [slots][4][tc]
    double *acc;       // [3][n] caller rows
    double *pot;       // [n] or null
    double *vel;       // [3][n] or null: fused closing half-kick v += half_dt * a
    int64_t n;
    double G;
    double half_dt;
};

// Parameters of the FP32-compensated acceleration + jerk kernel.
struct F32CJerkParams {
    const float *px, *py, *pz, *pm, *pvx, *pvy, *pvz;
    const float4 *chl;   // position centres (hi, lo) per tile
    const float4 *vchl;  // velocity centres (hi, lo) per tile
    const int32_t *perm;
    const ClusterDev *cl;
    const Item *items;
    int32_t n_items;
    int32_t tc;
    int *counters;
    double *partial;     // [slots][7][tc]
    double *acc;         // [3][n]
    double *jerk;        // [3][n]
    double *pot;         // [n] or null
    int64_t n;
    double G;
};

// Parameters of the plain FP64 kernel.
struct F64Params {
    const double *pos;      // [3][n]
    const double *mass;     // [n]
    const ClusterDev *cl;
    const int2 *blocks;     // per CTA: (cluster, first local i)
    double *acc, *pot, *vel;
    int64_t n;
    double G;
    double half_dt;
    const double *velin;  // [3][n]: with jerk != null, the velocities the jerk uses
    double *jerk;         // [3][n] or null
};

struct PackParams {
    const double *pos;  // [3][n]
    const double *mass;
    const int32_t *perm;
    const ClusterDev *cl;
    const int32_t *tile_cluster;  // [n_tiles]
    int32_t tc;
    int64_t n;
    float *px, *py, *pz, *pm;
    float4 *chl;
    // optional velocity half (jerk path): mean velocity per tile as a float
    // pair (vchl) and FP32 offsets from it; pads get velocity offset 0
    const double *vel = nullptr;  // [3][n]
    float *pvx = nullptr, *pvy = nullptr, *pvz = nullptr;
    float4 *vchl = nullptr;
};

// A run of at most kChunk consecutive rows inside one cluster (energy, bbox, keys).
constexpr int kChunk = 2048;
struct Chunk {
    int32_t cluster;
    int32_t pad;
    int64_t begin, end;  // caller rows [begin, end)
};

// Block time steps (block_sched.cu, block_force.cu).  One work item: an i-chunk of the active list
// (positions a0 .. a0 + na - 1, all in one cluster) against one j-range split.
struct SubItem {
    int32_t a0, na, cluster, chunk;
    int32_t jt0, jt1, split, nsplit;
    int32_t pbase, pad;
};

// Device-side scalars of the block-step scheduler.
// Block steps with at most kFewMax active particles take the few-particle
// kernel (j-parallel) instead of the i-chunk subset kernel.
constexpr int kFewMax = 32;
constexpr int kFewCtas = 152;

struct BlockScalars {
    double t_next;   // time of the current block step
    long long t_next_q;  // the same in units of dt_min
    double t_end;    // stop time (set by the host before each batch)
    long long t_end_q;  // the same in units of dt_min (follows t_end in memory: set together)
    int n_active, n_chunks, split, n_items;
    long long blocks, evals;  // block steps taken, single-particle evaluations
    int ticket_min, ticket_pack, ticket_few;  // last-CTA tickets (each reset by its last CTA)
    // particles per step level k (dt = dt_max 2^-k), kept by the corrector; the
    // smallest occupied step gives the next step's time
    int level[64];
    // few-particle path (F32C, n_active <= kFewMax): the clusters holding active
    // particles, their first active index and the prefix of their sizes
    int few, few_ncl;
    int few_cl[kFewMax], few_abeg[kFewMax], few_jbase[kFewMax + 1];
    // i-chunk size of this step and the work each subset kernel sees (F32C:
    // the CTAs with a range of units; the kernel not chosen reads 0 and
    // returns at once)
    int cs, n_items_small, n_items_large;
    // F32C: time of the tile frames' origins (units of dt_min), set by the
    // fresh pack
    long long frame_t0q;
    // F32C subset kernels: the step's work, n_units (i-chunk, j-tile) units in
    // unit order (clusters, their i-chunks, the j-tiles), split evenly over
    // n_workers CTAs (the plan's work_off holds each cluster's first unit)
    long long n_units;
    int n_workers;
};

// Subset acceleration + jerk kernel: base carries the j-set (the jerk path's
// packed predicted particles), perm (slot -> row) and the outputs (rows).
// Hermite corrector + next-step choice of the block scheme, applied where an
// active particle's acceleration and jerk become final (block_common.cuh).
// F32C block steps: the state the packing predictor reads, in j-set slot
// order and in FP32, relative to a frame per centre tile that moves at a
// constant velocity: its position at time t is c(t) = c0 + cv (t - t0), c0 in
// FP64, cv the tile's FP32 velocity centre (vchl), t0 the time of the last
// fresh pack (BlockScalars::frame_t0q), which sets c0 and cv from the rows
// (after a re-sort, at the start of each advance).  Each slot holds its
// particle's x_i - c(t_i) (a float pair, so that the predicted offset is
// rounded to FP32 once) and v_i - cv at the particle's own time t_i, and FP32
// copies of a_i and a'_i; the corrector rewrites them.  The predicted offset
// from the frame at t is then a short FP32 polynomial in t - t_i, and the tile
// centre the force kernels see, c(t), is a float pair (hi + lo) from FP64.
struct SlotMirror {
    float *xr, *xl, *vr;   // [3][n_pad] x_i - c(t_i) as a float pair (xr + xl), v_i - cv
    float *af, *jf;        // [3][n_pad]
    long long *tcq, *tq;   // [n_pad] t_i and t_i + dt_i in units of dt_min
    double *c0;            // [3][n_tiles] frame origins at t0
    const float4 *vchl;    // frame velocities: vchl[2 tile].xyz
    int tc, n_tiles;       // slots per tile, tiles
    int64_t n_pad;
};

struct BlockCorrect {
    const BlockScalars *sc;
    int *level;  // BlockScalars::level (the corrector moves particles between levels)
    SlotMirror m;  // m.xr == null: no mirror (FP64 path)
    double *t, *dt, *pos, *vel, *acc, *jerk, *pot;  // rows; acc, jerk: the particle's a0, j0
    long long *tq;
    int64_t n;
    double dt_max, dt_min, eta;
};

// Level of a power-of-two step h below dt_max: dt_max / h = 2^level (from the
// exponent fields, exact).
__host__ __device__ __forceinline__ int block_level(double h, double dt_max) {
    long long bh, bm;
    memcpy(&bh, &h, sizeof bh);
    memcpy(&bm, &dt_max, sizeof bm);
    return (int)((bm >> 52) & 0x7FF) - (int)((bh >> 52) & 0x7FF);
}

// Even split of the block-step subset kernels' work (F32C): n_units
// (i-chunk, j-tile) units in order, cut into n_ranges contiguous ranges, one
// per CTA; range r is [even_range_begin(r), even_range_begin(r + 1)).
__host__ __device__ __forceinline__ long long even_range_begin(long long r, long long n_units,
                                                              long long n_ranges) {
    return r * n_units / n_ranges;
}

// The range holding unit u (the last r with even_range_begin(r) <= u).
__host__ __device__ __forceinline__ long long even_range_of(long long u, long long n_units,
                                                           long long n_ranges) {
    return ((u + 1) * n_ranges - 1) / n_units;
}

// Partial slot of range r's part of an i-chunk whose first unit is uc and that
// other ranges share: 2r when the range starts in the chunk (its first
// i-chunk), 2r + 1 when it started before (the chunk is its last).
__host__ __device__ __forceinline__ long long even_range_slot(long long r, long long uc, long long n_units,
                                                             long long n_ranges) {
    return even_range_begin(r, n_units, n_ranges) >= uc ? 2 * r : 2 * r + 1;
}

// The step's plan (one thread, after the scan of the per-unit active counts;
// cluster c owns units [unit_first[c], unit_first[c + 1])): per-cluster active
// ranges and i-chunk counts, the regime, and the force pass's work.  F32C
// (work_off given): the (i-chunk, j-tile) units in unit order -- clusters,
// their i-chunks, the j-tiles -- cut into one contiguous range for each of up
// to `workers` CTAs (at least kMinUnits units a range, and a multiple of the
// SM count once there are that many, so that every SM holds as many ranges;
// work_off[c] = cluster c's first unit).  A static even split: every CTA
// gets the same work to within a unit, where a queue of (i-chunk, j-range)
// items handed out two rounds of 5-6 j-tiles and left SMs idle for the last
// ones.  FP64 path: queue items (i-chunk, j-range split), the split chosen so
// that the last round is fullest.
__host__ __device__ inline void plan_step(const int *__restrict__ unit_off, int total, int n_units,
                          const int32_t *__restrict__ unit_first, int ncl,
                          const ClusterDev *__restrict__ cl, int cs_small, int workers_small,
                          int max_split, int *__restrict__ act_begin, int *__restrict__ act_n,
                          int *__restrict__ ich_off, int *__restrict__ item_off, BlockScalars *sc,
                          int few_max, int cs_large, int workers_large, int large_min,
                          long long partial_cap, long long *__restrict__ work_off = nullptr, int sms = 1) {
    const bool even_units = work_off != nullptr;  // F32C: even ranges of units
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
    if (split < 1 || even_units) split = 1;
    // equal-cost items drain in ceil(items / workers) rounds: among the next few
    // split counts that fit the partial buffer, take the one whose last round
    // is fullest (the smaller on ties)
    if (chunks > 0 && !even_units) {
        // fullness of the last round, items / (workers * rounds), compared
        // exactly as fractions in integers (no FP64 division on this thread,
        // which every step waits for)
        const long long max_slots = partial_cap / (7LL * cs);
        long long best_items = 0, best_rounds = 1;
        int pick = split;
        for (int sp = split; sp <= split + 3 && sp <= max_split; ++sp) {
            const long long items = (long long)chunks * sp;
            if (sp > 1 && items > max_slots) break;
            const long long rounds = (items + workers - 1) / workers;
            if (items * best_rounds > best_items * rounds) {
                best_items = items;
                best_rounds = rounds;
                pick = sp;
            }
        }
        split = pick;
    }
    int items = 0;
    if (even_units) {
        constexpr long long kMinUnits = 2;  // bounds the partials summed per chunk
        long long w = 0;
        for (int c = 0; c < ncl; ++c) {
            work_off[c] = w;
            w += (long long)(ich_off[c + 1] - ich_off[c]) * cl[c].n_jt;
        }
        work_off[ncl] = w;
        long long nw = w / kMinUnits;
        if (nw > workers) nw = workers;
        if (nw > sms) nw -= nw % sms;  // every SM the same number of ranges
        if (nw < 1) nw = 1;
        sc->n_units = w;
        sc->n_workers = chunks > 0 ? (int)nw : 0;
    } else {
        for (int c = 0; c < ncl; ++c) {
            item_off[c] = items;
            const int sc_c = split < cl[c].n_jt ? split : (cl[c].n_jt > 0 ? cl[c].n_jt : 1);
            items += (ich_off[c + 1] - ich_off[c]) * sc_c;
        }
        item_off[ncl] = items;
    }
    sc->n_active = total;
    sc->n_chunks = chunks;
    sc->split = split;
    sc->n_items = items;
    sc->cs = cs;
    const int work = even_units ? sc->n_workers : items;  // what the chosen subset kernel sees
    sc->n_items_small = large ? 0 : work;
    sc->n_items_large = large ? work : 0;
    if (total > 0) {
        sc->blocks += 1;
        sc->evals += total;
    }
}

// The next block time (in units of dt_min) after a step at time tq_now that
// moved n_moved particles.  Every t_i is a multiple of its step dt_i with
// t_i <= t_now < t_i + dt_i, so min (t_i + dt_i) is the next multiple of the
// smallest occupied step; a step that moved nobody (past t_end, or the start)
// leaves the time pending.
__host__ __device__ __forceinline__ long long block_next_time_q(long long tq_now, int n_moved,
                                                                const int *level, double dt_max,
                                                                double dt_min) {
    if (n_moved == 0) return tq_now;
    const int kmax = block_level(dt_min, dt_max);
    int k = kmax;
    while (k > 0 && level[k] == 0) --k;
    const long long step_q = 1LL << (kmax - k);
    return (tq_now / step_q + 1) * step_q;
}

struct F32CSubsetParams {
    F32CJerkParams base;
    BlockCorrect corr;        // corr.sc == nullptr: store a1, j1, p1 instead
    const int32_t *act_slot;  // active list: j-set slot of each active particle
    const int *n_items;       // device count: the CTAs with a range of units
    // the plan, per cluster: first active index, active count, first i-chunk,
    // first (i-chunk, j-tile) unit; and the step's scalars (n_units, n_workers)
    const int *act_begin, *act_n, *ich_off;
    const long long *work_off;
    int ncl;
    const BlockScalars *sc;
    double *partial;          // [slots][7][block * p]
    int tcj;                  // j-set centre-tile size
    // low parts of the packed position offsets (px + pxl, ...), or null: the
    // few-particle pass then differences close pairs exactly
    const float *pxl, *pyl, *pzl;
};

struct BlockLaunch {
    int64_t n;
    int ncl, n_chunks, cs, workers, max_split, max_items;
    const Chunk *chunks;
    const int32_t *chunk_first;
    const ClusterDev *cl;
    double *t, *dt, *part;
    long long *tq;  // t_i + dt_i in units of dt_min (exact: steps are powers of two >= dt_min)
    double dt_min, dt_max;
    double *pos, *vel, *acc, *jerk, *xp, *vp;
    SlotMirror mirror;  // F32C: the packing predictor's slot-ordered state
    bool fresh;         // F32C: new tile frames and mirror from the rows (after a re-sort, ...)
    const double *mass;
    uint8_t *flag;  // per row (FP64) or per j-set slot (F32C)
    // per row chunk (FP64) or per centre tile (F32C): active counts, offsets
    int *cnt, *chunk_off, *act_begin, *act_n, *ich_off, *item_off;
    long long *work_off;  // F32C: per cluster, first (i-chunk, j-tile) unit of the step's work
    int32_t *act;
    SubItem *items;  // FP64 path: the work queue
    SubItem *info;   // FP64 path: per i-chunk: range, cluster, split count, partial base
    BlockScalars *sc;
    // F32C j-set geometry (px == nullptr on the FP64 path)
    const int32_t *perm, *tile_cluster, *tile_first;
    int tc, n_tiles;
    float *px, *py, *pz, *pm, *pvx, *pvy, *pvz;
    float *pxl, *pyl, *pzl;  // low parts of the position offsets (block steps)
    float4 *chl, *vchl;
    int few_max;  // 0 disables the few-particle path
    // second subset kernel for large active sets (cs_large == 0: none)
    int cs_large, workers_large, large_min;
    long long partial_cap;  // doubles in the subset kernels' split-partial buffer
    int sms;  // multiprocessors (the even split's range count is a multiple)
    unsigned long long *trace;  // F32C per-step trace (NBODY_FLAG_TRACE) or null
    int trace_cap;
};

cudaError_t launch_block_init(int64_t n, const double *acc, const double *jerk, double dt_max,
                              double dt_min, double eta_s, double *t, double *dt, long long *tq,
                              cudaStream_t s);
// t_next (FP64 path: integer min; F32C: from the level counts), prediction
// (+ the packed j-set for F32C), flags, counts and the plan (offsets, regime,
// and the force pass's work: F32C even ranges of units, FP64 queue items).
cudaError_t launch_block_prepare(const BlockLaunch &b, cudaStream_t s, int *kernels);
// NBODY_FLAG_TRACE: the end record of an advance call's last step, if no pack
// after it wrote one.
cudaError_t launch_block_trace_end(const BlockScalars *sc, unsigned long long *trace, int cap, cudaStream_t s);
// Ordered compaction of the active particles (rows, or j-set slots for F32C)
// and, on the FP64 path, the work queue.
cudaError_t launch_block_queue(const BlockLaunch &b, cudaStream_t s, int *kernels);
int subset_occupancy(int block, int p, int tj, int groups, int minb, bool eps_zero);
int subset_shapes(int *block, int *p, int *tj, int *groups, int *minb, int cap);
// The force pass's last kernel: the few-particle pass (all j of the active
// clusters in parallel, FP64 partials per CTA in few_part: kFewCtas * kFewMax
// * 7 doubles, summed in order by the last CTA) when the plan chose it, else
// the deterministic parallel sum of the subset kernels' split partials; both
// apply the epilogue and the corrector.
cudaError_t launch_subset_tail(int max_chunks, int max_cs, int max_ctas, const F32CSubsetParams &prm,
                               const int32_t *act, BlockScalars *sc, double *few_part, cudaStream_t s);
// Level counts of all particles and the first t_next (start of block stepping).
cudaError_t launch_block_levels(int64_t n, const double *dt, double dt_max, double dt_min,
                                const Chunk *chunks, int n_chunks, const long long *tq, double *part,
                                BlockScalars *sc, cudaStream_t s);
// block * groups threads per CTA (see SubsetKernel in block_force.cu).
cudaError_t launch_subset_f32c(int block, int p, int tj, int groups, int minb, bool eps_zero,
                               int grid, const F32CSubsetParams &prm, cudaStream_t s);
cudaError_t launch_subset_f64(int max_items, const double *xp, const double *vp, const double *mass,
                              const ClusterDev *cl, const SubItem *items, const int *n_items,
                              const int32_t *act, int64_t n, double G, double *acc, double *jerk,
                              double *pot, cudaStream_t s);
// The corrector as its own pass over the active list (the FP64 path; the F32C
// force kernels apply it in their epilogues).
cudaError_t launch_block_correct(const BlockCorrect &c, const int32_t *act, const double *a1,
                                 const double *j1, const double *p1, cudaStream_t s);


// ---- kernel launchers (all enqueue on `s`, return cudaGetLastError()) ----

// The F32C force kernel for tile shape (block, p, tj) compiled for minb resident
// CTAs per SM (0 = the first compiled variant); eps_zero selects the variant that
// gives coincident pairs zero force (needed when some eps == 0).  Returns
// cudaErrorNotSupported if the shape is not compiled.  `grid` CTAs run the
// persistent work loop.
cudaError_t launch_f32c(int block, int p, int tj, int minb, bool eps_zero, int grid,
                        const F32CParams &prm, cudaStream_t s);
// Maximum resident CTAs per SM of the given shape (0 if not compiled).
int f32c_occupancy(int block, int p, int tj, int minb, bool eps_zero);
// The minb of the variant that (block, p, tj, minb) selects (0 if none).
int f32c_resolve_minb(int block, int p, int tj, int minb, bool eps_zero);
// Compiled shapes: fills up to cap (block, p, tj, minb), returns the count.
int f32c_shapes(int *block, int *p, int *tj, int *minb, int cap);

cudaError_t launch_f64(int grid, const F64Params &prm, cudaStream_t s);
constexpr int kF64Block = 128;

// One CTA per centre tile; tc must be a positive multiple of 128.
cudaError_t launch_pack(int n_tiles, const PackParams &prm, cudaStream_t s);

// Acceleration + jerk kernel (forces_f32c_jerk.cuh), same conventions as launch_f32c.
cudaError_t launch_f32c_jerk(int block, int p, int tj, int minb, bool eps_zero, int grid,
                             const F32CJerkParams &prm, cudaStream_t s);
int f32c_jerk_occupancy(int block, int p, int tj, int minb, bool eps_zero);
int f32c_jerk_resolve_minb(int block, int p, int tj, int minb, bool eps_zero);
int f32c_jerk_shapes(int *block, int *p, int *tj, int *minb, int cap);

// Hermite predictor: xp = x + v dt + a dt^2/2 + j dt^3/6, vp = v + a dt + j dt^2/2.
cudaError_t launch_hermite_predict(int64_t n3, const double *pos, const double *vel,
                                   const double *acc, const double *jerk, double dt, double *xp,
                                   double *vp, cudaStream_t s);
// Hermite corrector: v1 = v + (a0 + a1) dt/2 + (j0 - j1) dt^2/12,
// x1 = x + (v + v1) dt/2 + (a0 - a1) dt^2/12; then acc <- a1, jerk <- j1.
cudaError_t launch_hermite_correct(int64_t n3, double *pos, double *vel, double *acc, double *jerk,
                                   const double *a1, const double *j1, double dt, cudaStream_t s);

cudaError_t launch_kick_drift(int64_t n3, double *pos, double *vel, const double *acc,
                              double half_dt, double dt, cudaStream_t s);

// Two-stage deterministic per-cluster reduction of K, W, P, L.
// part: double[n_chunks][8]; out: double[ncl][9] at out_base + (*counter) * ncl * 9
// when counter != null (the counter is then incremented), else at out_base.
cudaError_t launch_energy(const double *pos, const double *vel, const double *mass,
                          const double *pot, int64_t n, const Chunk *chunks, int n_chunks,
                          const int32_t *chunk_first, int ncl, double *part, double *out_base,
                          int *counter, cudaStream_t s);

// Morton reordering: fills perm[slot] for every real slot.  Clusters of at most
// kSmemSortMax particles are sorted one CTA per cluster in shared memory (then
// keys/vals/part/bbox are unused and may be null); otherwise keys/vals are
// scratch of sort_n (power of two >= n) entries, part double[n_chunks][6] and
// bbox double[ncl][6].
constexpr int64_t kSmemSortMax = 16384;
bool reorder_in_smem(int64_t max_cluster);
cudaError_t launch_reorder(const double *pos, int64_t n, const Chunk *chunks, int n_chunks,
                           const int32_t *chunk_first, int ncl, const ClusterDev *cl,
                           double *part, double *bbox, unsigned long long *keys, uint32_t *vals,
                           int64_t sort_n, int64_t max_cluster, int32_t *perm, cudaStream_t s,
                           int *launches);

// Sets *flag = 1 if any of the n3 + n values is not finite.
cudaError_t launch_check_finite(const double *acc, int64_t n3, const double *pot, int64_t n,
                                int *flag, cudaStream_t s);

}  // namespace nbody
