// nbody_abi.cu -- the C ABI of libnbody.so: contexts, work queue, staging of
// host buffers, CUDA-graph capture of leapfrog steps, profiling and the
// autotuner.  The arithmetic lives in the kernels; this file only plans and
// enqueues them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <queue>
#include <string>
#include <unordered_map>
#include <vector>

#include "nbody.h"
#include "nbody_internal.h"

using namespace nbody;

namespace {

constexpr int kProfSlots = 2;

struct GraphEntry {
    const void *pos, *vel, *mass, *acc, *pot, *diag, *jerk;
    int kind;  // 0 = KDK leapfrog step, 1 = Hermite step, 2 = block step
    uint64_t dt_bits;
    int reorder;  // variant: re-sort and, for block steps, fresh pack (see step_common)
    int slot;
    cudaGraphExec_t exec;
    int kernels;
    int steps;  // steps captured in the graph
};

// Block steps replayed without profiling events go kMultiSteps to a graph
// (fewer graph launches per step).
constexpr int kMultiSteps = 8;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Acceleration + jerk path: its own tile geometry, queue and packed positions
// and velocities (built on first use), plus the Hermite step's scratch.
struct JerkPath {
    bool built = false;
    nbody_tiles tiles{0, 0, 0, 0, 0};
    int tc = 0, grid = 0, n_items = 0, n_tiles = 0;
    int64_t n_pad = 0;
    ClusterDev *dcl = nullptr;
    int32_t *tile_cluster = nullptr;
    int32_t *tile_first = nullptr;  // [ncl + 1] first centre tile of each cluster
    Item *items = nullptr;
    int *counters = nullptr;
    double *partial = nullptr;
    float *px = nullptr, *py = nullptr, *pz = nullptr, *pm = nullptr;
    float *pvx = nullptr, *pvy = nullptr, *pvz = nullptr;
    float4 *chl = nullptr, *vchl = nullptr;
    int32_t *perm = nullptr;
    double *xp = nullptr, *vp = nullptr, *a1 = nullptr, *j1 = nullptr;
};

// Individual (block) time steps: per-particle times and steps, the device-side
// scheduler's scratch and the subset kernel's partial sums.
struct BlockState {
    bool started = false;
    double dt_max = 0.0, dt_min = 0.0, eta = 0.0;
    int cs = 0, workers = 1, max_split = 1, max_items = 0, max_chunks = 0;
    // Morton re-sorting follows simulated time here: once per reorder_every
    // multiples of dt_max, at the start of the next 16-step batch
    int64_t reorder_epoch = 0;
    bool reorder_pending = false;
    // F32C: the next step packs from the rows and sets new tile frames (after
    // a re-sort, and at the start of every advance: the rows are the caller's)
    bool fresh_pending = false;
    // subset kernel shapes (F32C; split holds the thread-group count): small
    // active sets, and large ones from large_min active particles on
    nbody_tiles sub{0, 0, 0, 0, 0}, sub_large{0, 0, 0, 0, 0};
    int cs_large = 0, workers_large = 0, large_min = 0;
    long long partial_cap = 0;
    double *t = nullptr, *dt = nullptr, *part = nullptr, *partial = nullptr, *p1 = nullptr;
    double *few_part = nullptr;  // few-particle path: kFewCtas * kFewMax * 7
    long long *tq = nullptr;     // t_i + dt_i in units of dt_min
    SlotMirror m{};  // F32C: the packing predictor's state in j-set slot order
    float *pxl = nullptr, *pyl = nullptr, *pzl = nullptr;  // F32C: low parts of the packed offsets
    uint8_t *flag = nullptr;
    int *cnt = nullptr, *chunk_off = nullptr, *act_begin = nullptr, *act_n = nullptr;
    int *ich_off = nullptr, *item_off = nullptr;
    long long *work_off = nullptr;
    unsigned long long *trace = nullptr;  // NBODY_FLAG_TRACE: NBODY_TRACE_CAP records of (time, count)
    int32_t *act = nullptr;
    SubItem *items = nullptr, *info = nullptr;
    BlockScalars *sc = nullptr;
};

}  // namespace

struct nbody_ctx {
    // configuration
    int64_t n = 0;
    int ncl = 1;
    int mode = NBODY_F32C;
    double G = 1.0;
    int reorder_every = 0;
    int flags = 0;
    std::vector<int64_t> off;
    std::vector<double> eps;
    int device = 0;
    int sms = 1;
    std::string gpu_name;
    bool eps_zero = false;
    int64_t max_cluster = 0;

    // F32C geometry
    nbody_tiles tiles{0, 0, 0, 0, 0};
    int tc = 0;
    int grid = 0;
    std::vector<ClusterDev> hcl;
    ClusterDev *dcl = nullptr;
    int64_t n_pad = 0;
    int n_tiles = 0;
    int32_t *tile_cluster = nullptr;
    int32_t *tile_first = nullptr;  // [ncl + 1] first centre tile of each cluster
    Item *items = nullptr;
    int n_items = 0;
    int *counters = nullptr;
    double *partial = nullptr;
    float *px = nullptr, *py = nullptr, *pz = nullptr, *pm = nullptr;
    float4 *chl = nullptr;
    int32_t *perm = nullptr;

    // F64
    int2 *blocks64 = nullptr;
    int n_blocks64 = 0;

    // chunks (energy, bbox, keys)
    Chunk *chunks = nullptr;
    int n_chunks = 0;
    int32_t *chunk_first = nullptr;
    double *epart = nullptr;
    double *edev = nullptr;
    int *diag_counter = nullptr;
    int *finite_flag = nullptr;

    // reorder
    double *bpart = nullptr, *bbox = nullptr;
    unsigned long long *keys = nullptr;
    uint32_t *vals = nullptr;
    int64_t sort_n = 0;
    int64_t evals = 0;

    // staging of host arrays
    DevBuf st_pos, st_vel, st_mass, st_acc, st_pot, st_diag, st_jerk;

    // acceleration + jerk path
    JerkPath jp;

    // block time steps
    BlockState bs;

    // graphs
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;

    // profiling
    cudaEvent_t ev[kProfSlots][2] = {};
    bool ev_pending[kProfSlots] = {};
    int ev_next = 0;
    double prof_ms = 0.0;
    int64_t prof_count = 0;

    int64_t launches = 0;
    int sticky = NBODY_OK;
    std::string msg;

    // device bytes held by the context and the cap on them (0 = none)
    int64_t dev_bytes = 0;
    int64_t cap_bytes = 0;
};

namespace {

int fail(nbody_ctx *c, int code, const std::string &what) {
    if (c) {
        if (c->sticky == NBODY_OK) c->sticky = code;
        c->msg = what;
    }
    return code;
}

int cuda_fail(nbody_ctx *c, cudaError_t e, const char *where) {
    cudaGetLastError();
    return fail(c, NBODY_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define NB_CUDA(call)                                                 \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);      \
    } while (0)

// Ledger of the device allocations of every context (pointer -> owner, bytes),
// so that frees made without the context at hand still update its total.
std::mutex g_ledger_mutex;
std::unordered_map<void *, std::pair<nbody_ctx *, size_t>> g_ledger;

// cudaMalloc of `bytes` for ctx, refused with NBODY_ENOMEM (before any CUDA
// call) when it would take the context past its allocation cap.
int ctx_malloc(nbody_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (ctx && ctx->cap_bytes > 0 && ctx->dev_bytes + (int64_t)bytes > ctx->cap_bytes)
        return fail(ctx, NBODY_ENOMEM,
                    "allocation cap: " + std::to_string(bytes) + " more bytes would exceed the cap of " +
                        std::to_string(ctx->cap_bytes) + " (" + std::to_string(ctx->dev_bytes) + " held)");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, NBODY_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    if (ctx) {
        std::lock_guard<std::mutex> lock(g_ledger_mutex);
        g_ledger[*p] = {ctx, bytes};
        ctx->dev_bytes += (int64_t)bytes;
    }
    return NBODY_OK;
}

void ctx_free(void *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_ledger_mutex);
        auto it = g_ledger.find(p);
        if (it != g_ledger.end()) {
            it->second.first->dev_bytes -= (int64_t)it->second.second;
            g_ledger.erase(it);
        }
    }
    cudaFree(p);
}

template <class T>
int dev_alloc(nbody_ctx *ctx, T **p, size_t count) {
    if (*p) {
        ctx_free(*p);
        *p = nullptr;
    }
    void *q = nullptr;
    const int rc = ctx_malloc(ctx, &q, std::max<size_t>(count * sizeof(T), 256));
    *p = static_cast<T *>(q);
    return rc;
}

template <class T>
void dev_free(T **p) {
    ctx_free(*p);
    *p = nullptr;
}

template <class T>
int upload(nbody_ctx *ctx, T **p, const std::vector<T> &h) {
    int rc = dev_alloc(ctx, p, h.size());
    if (rc) return rc;
    if (!h.empty()) NB_CUDA(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return NBODY_OK;
}

int64_t cluster_n(const nbody_ctx *c, int k) { return c->off[k + 1] - c->off[k]; }

// ------------------------------------------------------------------ geometry

// Makespan of greedy largest-first assignment of `cost` to `workers` queues,
// the way the persistent CTAs drain the work queue.
double lpt_makespan(std::vector<double> cost, int workers) {
    std::sort(cost.begin(), cost.end(), std::greater<double>());
    std::priority_queue<double, std::vector<double>, std::greater<double>> q;
    for (int w = 0; w < workers; ++w) q.push(0.0);
    for (double x : cost) {
        double t = q.top();
        q.pop();
        q.push(t + x);
    }
    double m = 0.0;
    while (!q.empty()) {
        m = std::max(m, q.top());
        q.pop();
    }
    return m;
}

struct Plan {
    std::vector<ClusterDev> cl;
    std::vector<int32_t> tile_cluster;
    std::vector<Item> items;
    int64_t n_pad = 0;
    int n_tiles = 0;
    int partial_slots = 0;
};

// Lay the clusters out in centre tiles of tc slots and cut every i-tile's
// j-range into `split` pieces (fewer if the cluster has fewer j-tiles).
// jfrac < 1 truncates every j-range (only used to shorten autotuner timings).
Plan make_plan(const nbody_ctx *c, int tc, int tj, int split, double jfrac = 1.0) {
    Plan pl;
    int64_t slot = 0;
    for (int k = 0; k < c->ncl; ++k) {
        const int64_t nk = cluster_n(c, k);
        ClusterDev d{};
        d.user_begin = c->off[k];
        d.n = (int32_t)nk;
        d.slot_begin = (int32_t)slot;
        d.n_jt = (int32_t)((nk + tj - 1) / tj);
        d.eps2 = c->eps[k] * c->eps[k];
        d.eps2f = (float)d.eps2;
        const int64_t nit = (nk + tc - 1) / tc;
        for (int64_t t = 0; t < nit; ++t) pl.tile_cluster.push_back(k);
        slot += nit * tc;
        pl.cl.push_back(d);
    }
    pl.n_pad = slot;
    pl.n_tiles = (int)(slot / tc);
    struct Costed {
        Item it;
        double cost;
    };
    std::vector<Costed> tmp;
    int pslot = 0;
    for (int k = 0; k < c->ncl; ++k) {
        const ClusterDev &d = pl.cl[k];
        if (d.n == 0) continue;
        const int nit = (d.n + tc - 1) / tc;
        const int sk = std::max(1, std::min(split, d.n_jt));
        for (int t = 0; t < nit; ++t) {
            const int tile = d.slot_begin / tc + t;
            const int pbase = sk > 1 ? pslot : 0;
            if (sk > 1) pslot += sk;
            for (int s = 0; s < sk; ++s) {
                Item it{};
                it.tile = tile;
                it.cluster = k;
                it.jt0 = (int32_t)((int64_t)s * d.n_jt / sk);
                it.jt1 = (int32_t)((int64_t)(s + 1) * d.n_jt / sk);
                if (jfrac < 1.0) {
                    const int len = std::max(1, (int)std::ceil((it.jt1 - it.jt0) * jfrac));
                    it.jt1 = it.jt0 + len;
                }
                it.split = s;
                it.nsplit = sk;
                it.pbase = pbase;
                const double cost = (double)(it.jt1 - it.jt0) * tj + 0.25 * tj + (sk > 1 ? 0.25 * tj : 0.0);
                tmp.push_back({it, cost});
            }
        }
    }
    std::stable_sort(tmp.begin(), tmp.end(),
                     [](const Costed &a, const Costed &b) { return a.cost > b.cost; });
    for (auto &x : tmp) pl.items.push_back(x.it);
    pl.partial_slots = pslot;
    return pl;
}

// Split count that minimises the modelled makespan on `workers` CTAs.  Every
// count up to 24 is a candidate (the one whose items fill whole rounds of the
// resident CTAs is often not a round number), then coarser ones.
int choose_split(const nbody_ctx *c, int tc, int tj, int workers) {
    int best = 1;
    double best_t = 0.0;
    static const int kCandidates[] = {1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 11, 12, 13, 14, 15, 16,
                                      17, 18, 19, 20, 21, 22, 23, 24, 28, 32, 40, 48, 64};
    for (int s : kCandidates) {
        Plan pl = make_plan(c, tc, tj, s);
        std::vector<double> cost;
        cost.reserve(pl.items.size());
        for (auto &it : pl.items)
            cost.push_back((double)(it.jt1 - it.jt0) * tj + 0.25 * tj + (it.nsplit > 1 ? 0.25 * tj : 0.0));
        const double t = lpt_makespan(cost, workers);
        if (s == 1 || t < best_t * 0.995) {
            best_t = t;
            best = s;
        }
        if ((int64_t)pl.items.size() > 64LL * workers) break;
    }
    return best;
}

nbody_tiles default_tiles(const nbody_ctx *c) {
    if (c->max_cluster >= 65536) return {256, 4, 1024, 0, 1};
    if (c->max_cluster >= 8192) return {128, 2, 256, 0, 4};
    return {64, 2, 128, 0, 8};
}

void free_f32c(nbody_ctx *ctx) {
    dev_free(&ctx->dcl);
    dev_free(&ctx->tile_cluster);
    dev_free(&ctx->items);
    dev_free(&ctx->counters);
    dev_free(&ctx->partial);
    dev_free(&ctx->px);
    dev_free(&ctx->py);
    dev_free(&ctx->pz);
    dev_free(&ctx->pm);
    dev_free(&ctx->chl);
    dev_free(&ctx->perm);
}

void drop_graphs(nbody_ctx *ctx) {
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
}

// (Re)build every F32C buffer for tile shape t.  jfrac < 1 only for timing.
int build_f32c(nbody_ctx *ctx, nbody_tiles t, double jfrac = 1.0) {
    t.ctas_per_sm = f32c_resolve_minb(t.block, t.p, t.tj, t.ctas_per_sm, ctx->eps_zero);
    const int occ = t.ctas_per_sm ? f32c_occupancy(t.block, t.p, t.tj, t.ctas_per_sm, ctx->eps_zero) : 0;
    if (occ <= 0)
        return fail(ctx, NBODY_EUNSUPPORTED,
                    "tile shape (" + std::to_string(t.block) + "," + std::to_string(t.p) + "," +
                        std::to_string(t.tj) + ") is not compiled");
    const int tc = t.block * t.p;
    const int workers = occ * ctx->sms;
    if (t.split <= 0) t.split = choose_split(ctx, tc, t.tj, workers);
    Plan pl = make_plan(ctx, tc, t.tj, t.split, jfrac);
    if (pl.n_pad >= (int64_t)1 << 31) return fail(ctx, NBODY_EINVAL, "padded size exceeds 2^31");
    drop_graphs(ctx);
    free_f32c(ctx);
    ctx->tiles = t;
    ctx->tc = tc;
    ctx->hcl = pl.cl;
    ctx->n_pad = pl.n_pad;
    ctx->n_tiles = pl.n_tiles;
    ctx->n_items = (int)pl.items.size();
    ctx->grid = std::min(ctx->n_items, workers);
    int rc;
    if ((rc = upload(ctx, &ctx->dcl, pl.cl))) return rc;
    if ((rc = upload(ctx, &ctx->tile_cluster, pl.tile_cluster))) return rc;
    if ((rc = upload(ctx, &ctx->items, pl.items))) return rc;
    if ((rc = dev_alloc(ctx, &ctx->counters, (size_t)ctx->n_tiles + 1))) return rc;
    NB_CUDA(cudaMemset(ctx->counters, 0, ((size_t)ctx->n_tiles + 1) * sizeof(int)));
    if ((rc = dev_alloc(ctx, &ctx->partial, (size_t)pl.partial_slots * 4 * tc))) return rc;
    for (float **p : {&ctx->px, &ctx->py, &ctx->pz, &ctx->pm})
        if ((rc = dev_alloc(ctx, p, (size_t)ctx->n_pad))) return rc;
    if ((rc = dev_alloc(ctx, &ctx->chl, (size_t)ctx->n_tiles * 2))) return rc;
    // identity permutation within each cluster, -1 on pads
    std::vector<int32_t> perm((size_t)ctx->n_pad, -1);
    for (const ClusterDev &d : pl.cl)
        for (int32_t l = 0; l < d.n; ++l) perm[(size_t)d.slot_begin + l] = (int32_t)(d.user_begin + l);
    if ((rc = upload(ctx, &ctx->perm, perm))) return rc;
    ctx->evals = 0;  // the next evaluation re-sorts if reordering is on
    return NBODY_OK;
}

int build_common(nbody_ctx *ctx) {
    std::vector<Chunk> ch;
    std::vector<int32_t> first;
    for (int k = 0; k < ctx->ncl; ++k) {
        first.push_back((int32_t)ch.size());
        for (int64_t b = ctx->off[k]; b < ctx->off[k + 1]; b += kChunk)
            ch.push_back({k, 0, b, std::min<int64_t>(b + kChunk, ctx->off[k + 1])});
    }
    first.push_back((int32_t)ch.size());
    ctx->n_chunks = (int)ch.size();
    int rc;
    if ((rc = upload(ctx, &ctx->chunks, ch))) return rc;
    if ((rc = upload(ctx, &ctx->chunk_first, first))) return rc;
    if ((rc = dev_alloc(ctx, &ctx->epart, (size_t)ctx->n_chunks * 8))) return rc;
    if ((rc = dev_alloc(ctx, &ctx->edev, (size_t)ctx->ncl * 9))) return rc;
    if ((rc = dev_alloc(ctx, &ctx->diag_counter, 1))) return rc;
    if ((rc = dev_alloc(ctx, &ctx->finite_flag, 1))) return rc;
    if (ctx->mode == NBODY_F64) {
        std::vector<int2> blocks;
        for (int k = 0; k < ctx->ncl; ++k)
            for (int64_t l = 0; l < cluster_n(ctx, k); l += kF64Block) blocks.push_back(make_int2(k, (int)l));
        ctx->n_blocks64 = (int)blocks.size();
        if ((rc = upload(ctx, &ctx->blocks64, blocks))) return rc;
        std::vector<ClusterDev> cl;
        for (int k = 0; k < ctx->ncl; ++k) {
            ClusterDev d{};
            d.user_begin = ctx->off[k];
            d.n = (int32_t)cluster_n(ctx, k);
            d.eps2 = ctx->eps[k] * ctx->eps[k];
            d.eps2f = (float)d.eps2;
            cl.push_back(d);
        }
        ctx->hcl = cl;
        if ((rc = upload(ctx, &ctx->dcl, cl))) return rc;
    }
    if (ctx->mode == NBODY_F32C && ctx->reorder_every > 0 && ctx->n > 0 &&
        !reorder_in_smem(ctx->max_cluster)) {
        int64_t s = 1;
        while (s < ctx->n) s <<= 1;
        ctx->sort_n = s;
        if ((rc = dev_alloc(ctx, &ctx->keys, (size_t)s))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->vals, (size_t)s))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->bpart, (size_t)ctx->n_chunks * 6))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->bbox, (size_t)ctx->ncl * 6))) return rc;
    }
    return NBODY_OK;
}

// ------------------------------------------------------------------ staging

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller array: the pointer itself, or a staging buffer
// (filled from the host when copy_in).
int resolve(nbody_ctx *ctx, const void *user, size_t bytes, DevBuf &st, bool copy_in,
            cudaStream_t s, void **out, bool *staged) {
    *staged = false;
    if (!user || bytes == 0) {
        *out = const_cast<void *>(user);
        return NBODY_OK;
    }
    if (is_device_ptr(user)) {
        *out = const_cast<void *>(user);
        return NBODY_OK;
    }
    if (st.bytes < bytes) {
        ctx_free(st.p);
        st.p = nullptr;
        st.bytes = 0;
        if (int rc = ctx_malloc(ctx, &st.p, bytes)) return rc;
        st.bytes = bytes;
        drop_graphs(ctx);
    }
    if (copy_in) NB_CUDA(cudaMemcpyAsync(st.p, user, bytes, cudaMemcpyHostToDevice, s));
    *out = st.p;
    *staged = true;
    return NBODY_OK;
}

int check_ptr(nbody_ctx *ctx, const void *p, const char *name, bool required) {
    if (!p) return required ? fail(ctx, NBODY_EINVAL, std::string(name) + " is NULL") : NBODY_OK;
    if (((uintptr_t)p) % 8 != 0) return fail(ctx, NBODY_EINVAL, std::string(name) + " is not 8-byte aligned");
    return NBODY_OK;
}

// ------------------------------------------------------------------ enqueue

struct Arrays {
    double *pos, *vel, *acc, *pot, *diag;
    const double *mass;
    double *jerk = nullptr;
};

int prof_drain(nbody_ctx *ctx, int slot) {
    if (!ctx->ev_pending[slot]) return NBODY_OK;
    NB_CUDA(cudaEventSynchronize(ctx->ev[slot][1]));
    float ms = 0.0f;
    NB_CUDA(cudaEventElapsedTime(&ms, ctx->ev[slot][0], ctx->ev[slot][1]));
    ctx->prof_ms += ms;
    ctx->prof_count += 1;
    ctx->ev_pending[slot] = false;
    return NBODY_OK;
}

int record(nbody_ctx *ctx, cudaEvent_t ev, cudaStream_t s, bool capturing) {
    if (capturing) NB_CUDA(cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal));
    else NB_CUDA(cudaEventRecord(ev, s));
    return NBODY_OK;
}

// Force evaluation: [reorder] + pack + queue reset + force kernel (F32C), or
// the FP64 kernel.  vel != null fuses the closing half-kick.  slot >= 0 brackets
// the force kernel with that profiling slot's events.
int enqueue_forces(nbody_ctx *ctx, const Arrays &a, double half_dt, bool reorder, int slot,
                   bool capturing, cudaStream_t s, int *kernels) {
    if (ctx->n == 0) return NBODY_OK;
    if (ctx->mode == NBODY_F32C) {
        if (reorder) {
            NB_CUDA(launch_reorder(a.pos, ctx->n, ctx->chunks, ctx->n_chunks, ctx->chunk_first,
                                   ctx->ncl, ctx->dcl, ctx->bpart, ctx->bbox, ctx->keys, ctx->vals,
                                   ctx->sort_n, ctx->max_cluster, ctx->perm, s, kernels));
        }
        PackParams pp{a.pos, a.mass, ctx->perm, ctx->dcl, ctx->tile_cluster, ctx->tc, ctx->n,
                      ctx->px, ctx->py, ctx->pz, ctx->pm, ctx->chl};
        NB_CUDA(launch_pack(ctx->n_tiles, pp, s));
        ++*kernels;
        NB_CUDA(cudaMemsetAsync(ctx->counters, 0, ((size_t)ctx->n_tiles + 1) * sizeof(int), s));
        F32CParams fp{};
        fp.px = ctx->px;
        fp.py = ctx->py;
        fp.pz = ctx->pz;
        fp.pm = ctx->pm;
        fp.chl = ctx->chl;
        fp.perm = ctx->perm;
        fp.cl = ctx->dcl;
        fp.items = ctx->items;
        fp.n_items = ctx->n_items;
        fp.tc = ctx->tc;
        fp.counters = ctx->counters;
        fp.partial = ctx->partial;
        fp.acc = a.acc;
        fp.pot = a.pot;
        fp.vel = a.vel;
        fp.n = ctx->n;
        fp.G = ctx->G;
        fp.half_dt = half_dt;
        int rc;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][0], s, capturing))) return rc;
        cudaError_t e = launch_f32c(ctx->tiles.block, ctx->tiles.p, ctx->tiles.tj,
                                    ctx->tiles.ctas_per_sm, ctx->eps_zero, ctx->grid, fp, s);
        if (e == cudaErrorNotSupported) return fail(ctx, NBODY_EUNSUPPORTED, "tile shape not compiled");
        NB_CUDA(e);
        ++*kernels;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][1], s, capturing))) return rc;
    } else {
        F64Params fp{a.pos, a.mass, ctx->dcl, ctx->blocks64, a.acc, a.pot, a.vel, ctx->n, ctx->G, half_dt};
        int rc;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][0], s, capturing))) return rc;
        NB_CUDA(launch_f64(ctx->n_blocks64, fp, s));
        ++*kernels;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][1], s, capturing))) return rc;
    }
    return NBODY_OK;
}

// One KDK step: kick + drift, forces with the closing kick fused, diagnostics.
int enqueue_step(nbody_ctx *ctx, const Arrays &a, double dt, bool reorder, int slot, bool capturing,
                 cudaStream_t s, int *kernels) {
    if (ctx->n == 0) return NBODY_OK;
    NB_CUDA(launch_kick_drift(3 * ctx->n, a.pos, a.vel, a.acc, 0.5 * dt, dt, s));
    ++*kernels;
    int rc = enqueue_forces(ctx, a, 0.5 * dt, reorder, slot, capturing, s, kernels);
    if (rc) return rc;
    if (a.diag) {
        NB_CUDA(launch_energy(a.pos, a.vel, a.mass, a.pot, ctx->n, ctx->chunks, ctx->n_chunks,
                              ctx->chunk_first, ctx->ncl, ctx->epart, a.diag, ctx->diag_counter, s));
        *kernels += ctx->n_chunks > 0 ? 2 : 1;
    }
    return NBODY_OK;
}

bool want_reorder(const nbody_ctx *ctx) {
    return ctx->mode == NBODY_F32C && ctx->reorder_every > 0 && ctx->evals % ctx->reorder_every == 0;
}

int next_slot(nbody_ctx *ctx) {
    if (!(ctx->flags & NBODY_FLAG_PROFILE)) return -1;
    const int slot = ctx->ev_next;
    ctx->ev_next = (ctx->ev_next + 1) % kProfSlots;
    int rc = prof_drain(ctx, slot);
    return rc ? rc - 1000 : slot;  // callers check < -1
}

int check_finite(nbody_ctx *ctx, const double *acc, const double *pot, cudaStream_t s) {
    if (!(ctx->flags & NBODY_FLAG_CHECK_FINITE) || ctx->n == 0) return NBODY_OK;
    NB_CUDA(cudaMemsetAsync(ctx->finite_flag, 0, sizeof(int), s));
    NB_CUDA(launch_check_finite(acc, 3 * ctx->n, pot, ctx->n, ctx->finite_flag, s));
    ctx->launches += 1;
    int h = 0;
    NB_CUDA(cudaMemcpyAsync(&h, ctx->finite_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    if (h) return fail(ctx, NBODY_ENONFINITE, "non-finite acceleration or potential");
    return NBODY_OK;
}

int guard(nbody_ctx *ctx) {
    if (!ctx) return NBODY_EINVAL;
    if (ctx->sticky != NBODY_OK) return NBODY_ESTATE;
    return NBODY_OK;
}

// ------------------------------------------------------------------ jerk path

void free_jerk(nbody_ctx *ctx) {
    JerkPath &j = ctx->jp;
    dev_free(&j.dcl);
    dev_free(&j.tile_cluster);
    dev_free(&j.tile_first);
    dev_free(&j.items);
    dev_free(&j.counters);
    dev_free(&j.partial);
    for (float **q : {&j.px, &j.py, &j.pz, &j.pm, &j.pvx, &j.pvy, &j.pvz}) dev_free(q);
    dev_free(&j.chl);
    dev_free(&j.vchl);
    dev_free(&j.perm);
    for (double **q : {&j.xp, &j.vp, &j.a1, &j.j1}) dev_free(q);
    j.built = false;
}

nbody_tiles default_jerk_tiles(const nbody_ctx *c, bool block_steps = false) {
    // block steps split j-ranges finely for small active sets and pack every
    // particle each step: 256-wide j-tiles and 256-particle centre tiles there
    // (measured faster at N = 102 400), 512-wide j-tiles for full evaluations
    if (c->max_cluster >= 65536) return block_steps ? nbody_tiles{128, 2, 256, 0, 2} : nbody_tiles{256, 2, 512, 0, 1};
    if (c->max_cluster >= 8192) return {128, 2, 256, 0, 2};
    return {64, 2, 128, 0, 4};
}

// Build the jerk path's geometry for tile shape t (F32C) and the Hermite scratch.
void free_block(nbody_ctx *ctx);

// (Re)builds the jerk path's j-set geometry; block-step state sized for the old
// geometry is dropped (nbody_block_start must be called again).
int build_jerk(nbody_ctx *ctx, nbody_tiles t, double jfrac = 1.0) {
    drop_graphs(ctx);
    free_block(ctx);
    free_jerk(ctx);
    JerkPath &j = ctx->jp;
    int rc;
    for (double **q : {&j.xp, &j.vp, &j.a1, &j.j1})
        if ((rc = dev_alloc(ctx, q, (size_t)3 * ctx->n))) return rc;
    if (ctx->mode == NBODY_F32C) {
        t.ctas_per_sm = f32c_jerk_resolve_minb(t.block, t.p, t.tj, t.ctas_per_sm, ctx->eps_zero);
        const int occ = t.ctas_per_sm
                            ? f32c_jerk_occupancy(t.block, t.p, t.tj, t.ctas_per_sm, ctx->eps_zero)
                            : 0;
        if (occ <= 0) return fail(ctx, NBODY_EUNSUPPORTED, "jerk tile shape is not compiled");
        const int tc = t.block * t.p;
        const int workers = occ * ctx->sms;
        if (t.split <= 0) t.split = choose_split(ctx, tc, t.tj, workers);
        Plan pl = make_plan(ctx, tc, t.tj, t.split, jfrac);
        if (pl.n_pad >= (int64_t)1 << 31) return fail(ctx, NBODY_EINVAL, "padded size exceeds 2^31");
        j.tiles = t;
        j.tc = tc;
        j.n_pad = pl.n_pad;
        j.n_tiles = pl.n_tiles;
        j.n_items = (int)pl.items.size();
        j.grid = std::min(j.n_items, workers);
        if ((rc = upload(ctx, &j.dcl, pl.cl))) return rc;
        if ((rc = upload(ctx, &j.tile_cluster, pl.tile_cluster))) return rc;
        std::vector<int32_t> tfirst(pl.cl.size() + 1, (int32_t)pl.n_tiles);
        for (size_t c = 0; c < pl.cl.size(); ++c) tfirst[c] = pl.cl[c].slot_begin / tc;
        if ((rc = upload(ctx, &j.tile_first, tfirst))) return rc;
        if ((rc = upload(ctx, &j.items, pl.items))) return rc;
        if ((rc = dev_alloc(ctx, &j.counters, (size_t)j.n_tiles + 1))) return rc;
        if ((rc = dev_alloc(ctx, &j.partial, (size_t)pl.partial_slots * 7 * tc))) return rc;
        for (float **q : {&j.px, &j.py, &j.pz, &j.pm, &j.pvx, &j.pvy, &j.pvz})
            if ((rc = dev_alloc(ctx, q, (size_t)j.n_pad))) return rc;
        if ((rc = dev_alloc(ctx, &j.chl, (size_t)j.n_tiles * 2))) return rc;
        if ((rc = dev_alloc(ctx, &j.vchl, (size_t)j.n_tiles * 2))) return rc;
        std::vector<int32_t> perm((size_t)j.n_pad, -1);
        for (const ClusterDev &d : pl.cl)
            for (int32_t l = 0; l < d.n; ++l) perm[(size_t)d.slot_begin + l] = (int32_t)(d.user_begin + l);
        if ((rc = upload(ctx, &j.perm, perm))) return rc;
    }
    j.built = true;
    ctx->evals = 0;
    return NBODY_OK;
}

int ensure_jerk(nbody_ctx *ctx) {
    if (ctx->jp.built) return NBODY_OK;
    return build_jerk(ctx, default_jerk_tiles(ctx));
}

F32CJerkParams jerk_params(const nbody_ctx *ctx, double *acc, double *jerk, double *pot) {
    const JerkPath &j = ctx->jp;
    F32CJerkParams fp{};
    fp.px = j.px; fp.py = j.py; fp.pz = j.pz; fp.pm = j.pm;
    fp.pvx = j.pvx; fp.pvy = j.pvy; fp.pvz = j.pvz;
    fp.chl = j.chl; fp.vchl = j.vchl; fp.perm = j.perm; fp.cl = j.dcl;
    fp.items = j.items; fp.n_items = j.n_items; fp.tc = j.tc;
    fp.counters = j.counters; fp.partial = j.partial;
    fp.acc = acc; fp.jerk = jerk; fp.pot = pot; fp.n = ctx->n; fp.G = ctx->G;
    return fp;
}

// Acceleration, jerk and potential at (pos, vel): [reorder] + pack + velocity
// pack + queue reset + jerk kernel (F32C), or the FP64 jerk kernel.
int enqueue_forces_jerk(nbody_ctx *ctx, const double *pos, const double *vel, const double *mass,
                        double *acc, double *jerk, double *pot, bool reorder, int slot,
                        bool capturing, cudaStream_t s, int *kernels) {
    if (ctx->n == 0) return NBODY_OK;
    JerkPath &j = ctx->jp;
    int rc;
    if (ctx->mode == NBODY_F32C) {
        if (reorder) {
            NB_CUDA(launch_reorder(pos, ctx->n, ctx->chunks, ctx->n_chunks, ctx->chunk_first, ctx->ncl,
                                   j.dcl, ctx->bpart, ctx->bbox, ctx->keys, ctx->vals, ctx->sort_n,
                                   ctx->max_cluster, j.perm, s, kernels));
        }
        PackParams pp{pos, mass, j.perm, j.dcl, j.tile_cluster, j.tc, ctx->n,
                      j.px, j.py, j.pz, j.pm, j.chl, vel, j.pvx, j.pvy, j.pvz, j.vchl};
        NB_CUDA(launch_pack(j.n_tiles, pp, s));
        *kernels += 1;
        NB_CUDA(cudaMemsetAsync(j.counters, 0, ((size_t)j.n_tiles + 1) * sizeof(int), s));
        const F32CJerkParams fp = jerk_params(ctx, acc, jerk, pot);
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][0], s, capturing))) return rc;
        cudaError_t e = launch_f32c_jerk(j.tiles.block, j.tiles.p, j.tiles.tj, j.tiles.ctas_per_sm,
                                         ctx->eps_zero, j.grid, fp, s);
        if (e == cudaErrorNotSupported) return fail(ctx, NBODY_EUNSUPPORTED, "jerk tile shape not compiled");
        NB_CUDA(e);
        ++*kernels;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][1], s, capturing))) return rc;
    } else {
        F64Params fp{pos, mass, ctx->dcl, ctx->blocks64, acc, pot, nullptr, ctx->n, ctx->G, 0.0,
                     vel, jerk};
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][0], s, capturing))) return rc;
        NB_CUDA(launch_f64(ctx->n_blocks64, fp, s));
        ++*kernels;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][1], s, capturing))) return rc;
    }
    return NBODY_OK;
}

// One Hermite step: predict, forces + jerks at the prediction, correct, diagnostics.
int enqueue_hermite_step(nbody_ctx *ctx, const Arrays &a, double dt, bool reorder, int slot,
                         bool capturing, cudaStream_t s, int *kernels) {
    if (ctx->n == 0) return NBODY_OK;
    JerkPath &j = ctx->jp;
    const int64_t n3 = 3 * ctx->n;
    NB_CUDA(launch_hermite_predict(n3, a.pos, a.vel, a.acc, a.jerk, dt, j.xp, j.vp, s));
    ++*kernels;
    int rc = enqueue_forces_jerk(ctx, j.xp, j.vp, a.mass, j.a1, j.j1, a.pot, reorder, slot,
                                 capturing, s, kernels);
    if (rc) return rc;
    NB_CUDA(launch_hermite_correct(n3, a.pos, a.vel, a.acc, a.jerk, j.a1, j.j1, dt, s));
    ++*kernels;
    if (a.diag) {
        NB_CUDA(launch_energy(a.pos, a.vel, a.mass, a.pot, ctx->n, ctx->chunks, ctx->n_chunks,
                              ctx->chunk_first, ctx->ncl, ctx->epart, a.diag, ctx->diag_counter, s));
        *kernels += ctx->n_chunks > 0 ? 2 : 1;
    }
    return NBODY_OK;
}

// ------------------------------------------------------------------ block steps

void free_block(nbody_ctx *ctx) {
    BlockState &b = ctx->bs;
    for (double **q : {&b.t, &b.dt, &b.part, &b.partial, &b.p1, &b.few_part}) dev_free(q);
    dev_free(&b.tq);
    for (float **q : {&b.m.xr, &b.m.xl, &b.m.vr, &b.m.af, &b.m.jf, &b.pxl, &b.pyl, &b.pzl}) dev_free(q);
    dev_free(&b.m.tcq);
    dev_free(&b.m.tq);
    dev_free(&b.m.c0);
    b.m = SlotMirror{};
    dev_free(&b.flag);
    for (int **q : {&b.cnt, &b.chunk_off, &b.act_begin, &b.act_n, &b.ich_off, &b.item_off}) dev_free(q);
    dev_free(&b.work_off);
    dev_free(&b.trace);
    dev_free(&b.act);
    dev_free(&b.items);
    dev_free(&b.info);
    dev_free(&b.sc);
    b.started = false;
}

int alloc_block(nbody_ctx *ctx) {
    BlockState &b = ctx->bs;
    free_block(ctx);
    int rc;
    const size_t n = (size_t)ctx->n, nc = (size_t)std::max(ctx->n_chunks, 1), ncl = (size_t)ctx->ncl;
    if (ctx->mode == NBODY_F32C) {
        // the subset kernels must stream the jerk geometry's j-tiles (same tj):
        // the small-set shape has several thread groups, the large-set one one
        int bl[16], pp[16], tj[16], gr[16], mb[16];
        const int ns = std::min(16, subset_shapes(bl, pp, tj, gr, mb, 16));
        b.sub = b.sub_large = nbody_tiles{0, 0, 0, 0, 0};
        for (int k = 0; k < ns; ++k) {
            if (tj[k] != ctx->jp.tiles.tj) continue;
            nbody_tiles &dst = gr[k] > 1 ? b.sub : b.sub_large;
            if (dst.block == 0) dst = nbody_tiles{bl[k], pp[k], tj[k], gr[k], mb[k]};
        }
        if (b.sub.block == 0 || b.sub_large.block == 0)
            return fail(ctx, NBODY_EUNSUPPORTED, "no subset kernel for the jerk tiles");
        b.cs = b.sub.block * b.sub.p;
        b.cs_large = b.sub_large.block * b.sub_large.p;
        const int occ = subset_occupancy(b.sub.block, b.sub.p, b.sub.tj, b.sub.split, b.sub.ctas_per_sm,
                                         ctx->eps_zero);
        const int occl = subset_occupancy(b.sub_large.block, b.sub_large.p, b.sub_large.tj,
                                          b.sub_large.split, b.sub_large.ctas_per_sm, ctx->eps_zero);
        if (occ <= 0 || occl <= 0) return fail(ctx, NBODY_EUNSUPPORTED, "subset kernel not loadable");
        b.workers = occ * ctx->sms;
        b.workers_large = occl * ctx->sms;
        b.large_min = 512;  // measured crossover at N = 102400
        b.max_split = 128;
        const int cs_min = std::min(b.cs, b.cs_large), cs_max = std::max(b.cs, b.cs_large);
        const int w_max = std::max(b.workers, b.workers_large);
        b.max_chunks = (int)(ctx->n / cs_min) + ctx->ncl + 1;
        // the plan's split count: chunks * split <= 2 * workers, plus up to 3
        // more splits per chunk to even out the last round
        b.max_items = 2 * w_max + 4 * b.max_chunks;
        // room for 2 partial slots per worker, or up to 4 per large-set i-chunk
        // (the plan may split every chunk to even out the last round), at most
        // 256 MiB beyond the former
        const long long base_cap = 2LL * w_max * 7 * cs_max;
        const long long big_cap = 4LL * ((long long)(ctx->n / b.cs_large) + ctx->ncl + 1) * 7 * b.cs_large;
        b.partial_cap = std::max(base_cap, std::min(big_cap, base_cap + (256LL << 20) / 8));
        if ((rc = dev_alloc(ctx, &b.partial, (size_t)b.partial_cap))) return rc;
        if ((rc = dev_alloc(ctx, &b.few_part, (size_t)kFewCtas * kFewMax * 7))) return rc;
    } else {
        b.cs = kF64Block;
        b.workers = 1;
        b.max_split = 1;
        b.max_chunks = std::max(ctx->n_blocks64, 1);
        b.max_items = b.max_chunks;
    }
    // flags per row (FP64) or per j-set slot (F32C); counts per row chunk or per tile
    const bool f32c = ctx->mode == NBODY_F32C;
    const size_t nflag = f32c ? (size_t)ctx->jp.n_pad : n;
    const size_t nunit = f32c ? (size_t)std::max(ctx->jp.n_tiles, 1) : nc;
    for (double **q : {&b.t, &b.dt, &b.p1})
        if ((rc = dev_alloc(ctx, q, n))) return rc;
    if ((rc = dev_alloc(ctx, &b.tq, n))) return rc;
    if (f32c) {
        const size_t np = (size_t)ctx->jp.n_pad;
        for (float **q : {&b.m.xr, &b.m.xl, &b.m.vr, &b.m.af, &b.m.jf})
            if ((rc = dev_alloc(ctx, q, 3 * np))) return rc;
        for (float **q : {&b.pxl, &b.pyl, &b.pzl})
            if ((rc = dev_alloc(ctx, q, np))) return rc;
        if ((rc = dev_alloc(ctx, &b.m.tcq, np)) || (rc = dev_alloc(ctx, &b.m.tq, np))) return rc;
        if ((rc = dev_alloc(ctx, &b.m.c0, 3 * (size_t)std::max(ctx->jp.n_tiles, 1)))) return rc;
        b.m.vchl = ctx->jp.vchl;
        b.m.tc = ctx->jp.tc;
        b.m.n_tiles = ctx->jp.n_tiles;
        b.m.n_pad = (int64_t)np;
    }
    if ((rc = dev_alloc(ctx, &b.part, nc))) return rc;
    if ((rc = dev_alloc(ctx, &b.flag, nflag))) return rc;
    for (int **q : {&b.cnt, &b.chunk_off})
        if ((rc = dev_alloc(ctx, q, nunit))) return rc;
    for (int **q : {&b.act_begin, &b.act_n, &b.ich_off, &b.item_off})
        if ((rc = dev_alloc(ctx, q, ncl + 1))) return rc;
    if (f32c && (rc = dev_alloc(ctx, &b.work_off, ncl + 1))) return rc;
    if (f32c && (ctx->flags & NBODY_FLAG_TRACE)) {
        if ((rc = dev_alloc(ctx, &b.trace, 2 * (size_t)NBODY_TRACE_CAP))) return rc;
        NB_CUDA(cudaMemset(b.trace, 0, 2 * (size_t)NBODY_TRACE_CAP * sizeof(unsigned long long)));
    }
    if ((rc = dev_alloc(ctx, &b.act, n))) return rc;
    if (!f32c) {  // the FP64 path's work queue (the F32C plan cuts even ranges of units)
        if ((rc = dev_alloc(ctx, &b.items, (size_t)b.max_items))) return rc;
        if ((rc = dev_alloc(ctx, &b.info, (size_t)b.max_chunks))) return rc;
    }
    if ((rc = dev_alloc(ctx, &b.sc, 1))) return rc;
    NB_CUDA(cudaMemset(b.sc, 0, sizeof(BlockScalars)));
    return NBODY_OK;
}

BlockLaunch block_launch(nbody_ctx *ctx, const Arrays &a) {
    BlockState &bs = ctx->bs;
    JerkPath &j = ctx->jp;
    BlockLaunch b{};
    b.n = ctx->n;
    b.ncl = ctx->ncl;
    b.n_chunks = ctx->n_chunks;
    b.cs = bs.cs;
    b.workers = bs.workers;
    b.max_split = bs.max_split;
    b.max_items = bs.max_items;
    b.chunks = ctx->chunks;
    b.chunk_first = ctx->chunk_first;
    b.cl = ctx->mode == NBODY_F32C ? j.dcl : ctx->dcl;
    b.t = bs.t;
    b.dt = bs.dt;
    b.tq = bs.tq;
    b.mirror = bs.m;
    b.dt_min = bs.dt_min;
    b.dt_max = bs.dt_max;
    b.part = bs.part;
    b.pos = a.pos;
    b.vel = a.vel;
    b.acc = a.acc;
    b.jerk = a.jerk;
    b.xp = j.xp;
    b.vp = j.vp;
    b.flag = bs.flag;
    b.cnt = bs.cnt;
    b.chunk_off = bs.chunk_off;
    b.act_begin = bs.act_begin;
    b.act_n = bs.act_n;
    b.ich_off = bs.ich_off;
    b.item_off = bs.item_off;
    b.work_off = bs.work_off;
    b.act = bs.act;
    b.items = bs.items;
    b.info = bs.info;
    b.sc = bs.sc;
    b.mass = a.mass;
    if (ctx->mode == NBODY_F32C) {
        b.perm = j.perm;
        b.tile_cluster = j.tile_cluster;
        b.tile_first = j.tile_first;
        b.tc = j.tc;
        b.n_tiles = j.n_tiles;
        b.px = j.px; b.py = j.py; b.pz = j.pz; b.pm = j.pm;
        b.pxl = bs.pxl; b.pyl = bs.pyl; b.pzl = bs.pzl;
        b.pvx = j.pvx; b.pvy = j.pvy; b.pvz = j.pvz;
        b.chl = j.chl; b.vchl = j.vchl;
        b.few_max = kFewMax;
        b.cs_large = bs.cs_large;
        b.workers_large = bs.workers_large;
        b.large_min = bs.large_min;
        b.partial_cap = bs.partial_cap;
        b.sms = ctx->sms;
        b.trace = bs.trace;
        b.trace_cap = NBODY_TRACE_CAP;
    }
    return b;
}

// One block step (see block_sched.cu, block_force.cu): schedule, predict, pack the predicted j-set,
// forces + jerks of the active subset, correct and re-step the active ones.
int enqueue_block_step(nbody_ctx *ctx, const Arrays &a, bool reorder, bool fresh, int slot, bool capturing,
                       cudaStream_t s, int *kernels) {
    if (ctx->n == 0) return NBODY_OK;
    BlockState &bs = ctx->bs;
    JerkPath &j = ctx->jp;
    BlockLaunch b = block_launch(ctx, a);
    b.fresh = fresh || reorder;
    int rc;
    if (ctx->mode == NBODY_F32C && reorder)
        NB_CUDA(launch_reorder(a.pos, ctx->n, ctx->chunks, ctx->n_chunks, ctx->chunk_first, ctx->ncl, j.dcl,
                               ctx->bpart, ctx->bbox, ctx->keys, ctx->vals, ctx->sort_n, ctx->max_cluster,
                               j.perm, s, kernels));
    NB_CUDA(launch_block_prepare(b, s, kernels));
    NB_CUDA(launch_block_queue(b, s, kernels));
    BlockCorrect corr{};
    corr.sc = bs.sc;
    corr.level = bs.sc->level;
    corr.m = bs.m;  // empty on the FP64 path
    corr.t = bs.t;
    corr.dt = bs.dt;
    corr.tq = bs.tq;
    corr.pos = a.pos;
    corr.vel = a.vel;
    corr.acc = a.acc;
    corr.jerk = a.jerk;
    corr.pot = a.pot;
    corr.n = ctx->n;
    corr.dt_max = bs.dt_max;
    corr.dt_min = bs.dt_min;
    corr.eta = bs.eta;
    if (ctx->mode == NBODY_F32C) {
        // the force kernels' epilogues apply the corrector (no separate pass)
        F32CSubsetParams q{};
        q.base = jerk_params(ctx, j.a1, j.j1, bs.p1);
        q.corr = corr;
        q.act_slot = bs.act;
        q.n_items = &bs.sc->n_items;
        q.act_begin = bs.act_begin;
        q.act_n = bs.act_n;
        q.ich_off = bs.ich_off;
        q.work_off = bs.work_off;
        q.ncl = ctx->ncl;
        q.sc = bs.sc;
        q.partial = bs.partial;
        q.tcj = j.tc;
        q.pxl = bs.pxl;
        q.pyl = bs.pyl;
        q.pzl = bs.pzl;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][0], s, capturing))) return rc;
        q.n_items = &bs.sc->n_items_small;
        NB_CUDA(launch_subset_f32c(bs.sub.block, bs.sub.p, bs.sub.tj, bs.sub.split,
                                   bs.sub.ctas_per_sm, ctx->eps_zero, bs.workers, q, s));
        q.n_items = &bs.sc->n_items_large;
        NB_CUDA(launch_subset_f32c(bs.sub_large.block, bs.sub_large.p, bs.sub_large.tj, bs.sub_large.split,
                                   bs.sub_large.ctas_per_sm, ctx->eps_zero, bs.workers_large, q, s));
        // few-particle pass or split-partial sum, whichever the plan chose
        NB_CUDA(launch_subset_tail(bs.max_chunks, std::max(bs.cs, bs.cs_large), 4 * ctx->sms, q, bs.act, bs.sc,
                                   bs.few_part, s));
        *kernels += 3;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][1], s, capturing))) return rc;
    } else {
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][0], s, capturing))) return rc;
        NB_CUDA(launch_subset_f64(bs.max_items, j.xp, j.vp, a.mass, ctx->dcl, bs.items,
                                  &bs.sc->n_items, bs.act, ctx->n, ctx->G, j.a1, j.j1, bs.p1, s));
        ++*kernels;
        if (slot >= 0 && (rc = record(ctx, ctx->ev[slot][1], s, capturing))) return rc;
        NB_CUDA(launch_block_correct(corr, bs.act, j.a1, j.j1, bs.p1, s));
        ++*kernels;
    }
    return NBODY_OK;
}

// ------------------------------------------------------------------ autotuner

std::string tune_key(const nbody_ctx *ctx) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%d|%d|%d|%lld|%d|%lld", ctx->gpu_name.c_str(), ctx->sms, ctx->mode,
             (int)ctx->eps_zero, (long long)ctx->n, ctx->ncl, (long long)ctx->max_cluster);
    std::string k(buf);
    for (char &ch : k)
        if (ch == ' ') ch = '_';
    return k;
}

bool tune_cache_lookup(const nbody_ctx *ctx, nbody_tiles *t) {
    const char *path = getenv("NBODY_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    const std::string key = tune_key(ctx);
    char kbuf[512];
    int b, p, tj, s, m;
    double ms;
    bool found = false;
    while (fscanf(f, "%511s %d %d %d %d %d %lf", kbuf, &b, &p, &tj, &s, &m, &ms) == 7)
        if (key == kbuf) {
            *t = {b, p, tj, s, m};
            found = true;
        }
    fclose(f);
    return found;
}

void tune_cache_store(const nbody_ctx *ctx, nbody_tiles t, double ms) {
    const char *path = getenv("NBODY_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %.6f\n", tune_key(ctx).c_str(), t.block, t.p, t.tj, t.split,
            t.ctas_per_sm, ms);
    fclose(f);
}

// Fill the packed arrays with a synthetic uniform cube per cluster (the force
// kernel's cost does not depend on the values, only on the shape).
__global__ void tune_fill_kernel(float *px, float *py, float *pz, float *pm, int64_t n_pad) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_pad;
         q += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)q * 2654435761u;
        px[q] = ((h >> 8) & 1023) / 1024.0f - 0.5f;
        h = h * 2246822519u + 374761393u;
        py[q] = ((h >> 8) & 1023) / 1024.0f - 0.5f;
        h = h * 3266489917u + 668265263u;
        pz[q] = ((h >> 8) & 1023) / 1024.0f - 0.5f;
        pm[q] = 1.0e-3f;
    }
}

// Time one tile shape: build its geometry (j-ranges scaled by jfrac), fill the
// packed arrays with a synthetic cube, best of `reps` timed launches (after one
// warm-up).  Returns the time in ms, or a negative status.
double time_shape(nbody_ctx *ctx, nbody_tiles t, double jfrac, int reps, double *acc, cudaEvent_t e0,
                  cudaEvent_t e1, cudaStream_t s, int *rc) {
    if ((*rc = build_f32c(ctx, t, jfrac))) return -1.0;
    tune_fill_kernel<<<256, 256, 0, s>>>(ctx->px, ctx->py, ctx->pz, ctx->pm, ctx->n_pad);
    if (cudaMemsetAsync(ctx->chl, 0, (size_t)ctx->n_tiles * 2 * sizeof(float4), s) != cudaSuccess) {
        *rc = cuda_fail(ctx, cudaGetLastError(), "tuner memset");
        return -1.0;
    }
    float best = 1e30f;
    for (int rep = 0; rep <= reps; ++rep) {
        F32CParams fp{};
        fp.px = ctx->px; fp.py = ctx->py; fp.pz = ctx->pz; fp.pm = ctx->pm;
        fp.chl = ctx->chl; fp.perm = ctx->perm; fp.cl = ctx->dcl;
        fp.items = ctx->items; fp.n_items = ctx->n_items; fp.tc = ctx->tc;
        fp.counters = ctx->counters; fp.partial = ctx->partial;
        fp.acc = acc; fp.pot = acc + 3 * ctx->n; fp.vel = nullptr; fp.n = ctx->n; fp.G = 1.0;
        cudaError_t e = cudaMemsetAsync(ctx->counters, 0, ((size_t)ctx->n_tiles + 1) * sizeof(int), s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess)
            e = launch_f32c(ctx->tiles.block, ctx->tiles.p, ctx->tiles.tj, ctx->tiles.ctas_per_sm,
                            ctx->eps_zero, ctx->grid, fp, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            *rc = cuda_fail(ctx, e, "tuner launch");
            return -1.0;
        }
        ctx->launches += 1;
        if (rep > 0) best = std::min(best, ms);
    }
    return best;
}

// Two rounds: every compiled shape (and three split counts) on a short proxy
// (j-ranges truncated to ~1e11 pairs), then the three fastest again on a proxy
// four times longer; the fastest of those is kept and cached.
int run_tuner(nbody_ctx *ctx, cudaStream_t s) {
    if (ctx->mode != NBODY_F32C || ctx->n == 0) return NBODY_OK;
    int blocks[64], ps[64], tjs[64], mbs[64];
    const int ns = std::min(64, f32c_shapes(blocks, ps, tjs, mbs, 64));
    double total_pairs = 0.0;
    for (int k = 0; k < ctx->ncl; ++k) total_pairs += (double)cluster_n(ctx, k) * cluster_n(ctx, k);
    const double jfrac = std::min(1.0, 1.0e11 / std::max(total_pairs, 1.0));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NB_CUDA(cudaEventCreate(&e0));
    if (cudaError_t e = cudaEventCreate(&e1)) {
        cudaEventDestroy(e0);
        return cuda_fail(ctx, e, "cudaEventCreate");
    }
    double *acc = nullptr;
    if (int rc0 = dev_alloc(ctx, &acc, (size_t)ctx->n * 4)) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc0;
    }
    std::vector<std::pair<double, nbody_tiles>> timed;
    int rc = NBODY_OK;
    for (int c = 0; c < ns && rc == NBODY_OK; ++c) {
        nbody_tiles t{blocks[c], ps[c], tjs[c], 0, mbs[c]};
        if ((int64_t)t.block * t.p > 2 * std::max<int64_t>(ctx->max_cluster, 128)) continue;
        const int occ = f32c_occupancy(t.block, t.p, t.tj, t.ctas_per_sm, ctx->eps_zero);
        const int base = choose_split(ctx, t.block * t.p, t.tj, occ * ctx->sms);
        for (int sv = 0; sv < 3 && rc == NBODY_OK; ++sv) {
            nbody_tiles tt = t;
            tt.split = sv == 0 ? base : sv == 1 ? base * 2 : std::max(1, base / 2);
            if (sv > 0 && tt.split == base) continue;
            const double ms = time_shape(ctx, tt, jfrac, 2, acc, e0, e1, s, &rc);
            if (rc == NBODY_OK) timed.push_back({ms, ctx->tiles});
        }
    }
    nbody_tiles best{0, 0, 0, 0, 0};
    double best_ms = 1e30;
    if (rc == NBODY_OK && !timed.empty()) {
        std::stable_sort(timed.begin(), timed.end(),
                         [](const std::pair<double, nbody_tiles> &x, const std::pair<double, nbody_tiles> &y) {
                             return x.first < y.first;
                         });
        // the three best again on a longer run: the full evaluation up to 2e12
        // pairs (a few seconds), else 4x the first proxy
        const double jfrac2 = std::min(1.0, std::max(4.0 * jfrac, 2.0e12 / std::max(total_pairs, 1.0)));
        for (size_t k = 0; k < std::min<size_t>(3, timed.size()) && rc == NBODY_OK; ++k) {
            const double ms = jfrac2 > jfrac ? time_shape(ctx, timed[k].second, jfrac2, 2, acc, e0, e1, s, &rc)
                                             : timed[k].first;
            if (rc == NBODY_OK && ms < best_ms) {
                best_ms = ms;
                best = timed[k].second;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(&acc);
    if (rc) return rc;
    if (best.block == 0) return fail(ctx, NBODY_EUNSUPPORTED, "autotuner found no usable shape");
    if ((rc = build_f32c(ctx, best))) return rc;
    tune_cache_store(ctx, best, best_ms);
    return NBODY_OK;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

const char *nbody_strerror(int status) {
    switch (status) {
        case NBODY_OK: return "success";
        case NBODY_EINVAL: return "invalid argument";
        case NBODY_ENOMEM: return "out of memory";
        case NBODY_ECUDA: return "CUDA runtime error";
        case NBODY_ENONFINITE: return "non-finite result";
        case NBODY_ETIMEOUT: return "device wait timed out";
        case NBODY_ESTATE: return "context is in an error state";
        case NBODY_EUNSUPPORTED: return "unsupported tile shape";
        case NBODY_ETOOBIG: return "n exceeds NBODY_NOALLOC_MAX_N, the fixed scratch of nbody_forces_noalloc";
        default: return "unknown status";
    }
}

const char *nbody_last_error_message(const nbody_ctx *ctx) { return ctx ? ctx->msg.c_str() : ""; }

int nbody_tiles_supported(nbody_tiles *out, int cap) {
    int b[64], p[64], t[64], m[64];
    const int n = f32c_shapes(b, p, t, m, 64);
    for (int k = 0; k < n && k < cap && out; ++k) out[k] = {b[k], p[k], t[k], 0, m[k]};
    return n;
}

void nbody_destroy(nbody_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    cudaGetLastError();
    drop_graphs(ctx);
    free_f32c(ctx);
    free_jerk(ctx);
    free_block(ctx);
    dev_free(&ctx->blocks64);
    dev_free(&ctx->chunks);
    dev_free(&ctx->chunk_first);
    dev_free(&ctx->epart);
    dev_free(&ctx->edev);
    dev_free(&ctx->diag_counter);
    dev_free(&ctx->finite_flag);
    dev_free(&ctx->bpart);
    dev_free(&ctx->bbox);
    dev_free(&ctx->keys);
    dev_free(&ctx->vals);
    for (DevBuf *b : {&ctx->st_pos, &ctx->st_vel, &ctx->st_mass, &ctx->st_acc, &ctx->st_pot,
                      &ctx->st_diag, &ctx->st_jerk})
        ctx_free(b->p);
    for (int s = 0; s < kProfSlots; ++s)
        for (int k = 0; k < 2; ++k)
            if (ctx->ev[s][k]) cudaEventDestroy(ctx->ev[s][k]);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
}

int nbody_init(nbody_ctx **out, const nbody_config *cfg, void *stream) {
    if (!out) return NBODY_EINVAL;
    *out = nullptr;
    if (!cfg) return NBODY_EINVAL;
    if (cfg->n_total < 0 || cfg->n_total > ((int64_t)1 << 30)) return NBODY_EINVAL;
    if (cfg->n_clusters < 1 || cfg->n_clusters > (1 << 24)) return NBODY_EINVAL;
    if (cfg->mode != NBODY_F64 && cfg->mode != NBODY_F32C) return NBODY_EINVAL;
    if (!cfg->eps || !std::isfinite(cfg->G) || cfg->reorder_every < 0) return NBODY_EINVAL;
    if (cfg->max_device_bytes < 0) return NBODY_EINVAL;
    if (cfg->n_clusters > 1 && !cfg->cluster_offsets) return NBODY_EINVAL;
    nbody_ctx *ctx = new nbody_ctx();
    ctx->n = cfg->n_total;
    ctx->ncl = cfg->n_clusters;
    ctx->mode = cfg->mode;
    ctx->G = cfg->G;
    ctx->reorder_every = cfg->reorder_every;
    ctx->flags = cfg->flags;
    ctx->cap_bytes = cfg->max_device_bytes;
    ctx->off.assign(cfg->n_clusters + 1, 0);
    if (cfg->cluster_offsets) {
        for (int k = 0; k <= cfg->n_clusters; ++k) ctx->off[k] = cfg->cluster_offsets[k];
    } else {
        ctx->off[1] = cfg->n_total;
    }
    bool ok = ctx->off[0] == 0 && ctx->off[ctx->ncl] == ctx->n;
    for (int k = 0; k < ctx->ncl && ok; ++k) ok = ctx->off[k + 1] >= ctx->off[k];
    ctx->eps.assign(cfg->eps, cfg->eps + cfg->n_clusters);
    for (double e : ctx->eps) ok = ok && std::isfinite(e) && e >= 0.0;
    if (!ok) {
        delete ctx;
        return NBODY_EINVAL;
    }
    for (int k = 0; k < ctx->ncl; ++k) {
        ctx->max_cluster = std::max(ctx->max_cluster, cluster_n(ctx, k));
        if ((float)(ctx->eps[k] * ctx->eps[k]) == 0.0f) ctx->eps_zero = true;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = NBODY_OK;
    do {
        cudaDeviceProp prop;
        cudaError_t e;
        if ((e = cudaGetDevice(&ctx->device)) != cudaSuccess ||
            (e = cudaGetDeviceProperties(&prop, ctx->device)) != cudaSuccess) {
            rc = cuda_fail(ctx, e, "device query");
            break;
        }
        ctx->sms = prop.multiProcessorCount;
        ctx->gpu_name = prop.name;
        if ((e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
            rc = cuda_fail(ctx, e, "stream create");
            break;
        }
        for (int sl = 0; sl < kProfSlots && rc == NBODY_OK; ++sl)
            for (int k = 0; k < 2; ++k)
                if ((e = cudaEventCreate(&ctx->ev[sl][k])) != cudaSuccess) rc = cuda_fail(ctx, e, "event create");
        if (rc) break;
        if ((rc = build_common(ctx))) break;
        if (ctx->mode == NBODY_F32C) {
            nbody_tiles t = cfg->tiles;
            const bool forced = t.block != 0 || t.p != 0 || t.tj != 0;
            if (!forced) {
                nbody_tiles cached;
                if (tune_cache_lookup(ctx, &cached)) t = cached;
                else if (cfg->flags & NBODY_FLAG_AUTOTUNE) t = {0, 0, 0, -1, 0};
                else {
                    t = default_tiles(ctx);
                    t.split = cfg->tiles.split;
                    if (cfg->tiles.ctas_per_sm) t.ctas_per_sm = cfg->tiles.ctas_per_sm;
                }
            }
            if (t.split == -1) {
                if ((rc = build_f32c(ctx, default_tiles(ctx)))) break;
                if ((rc = run_tuner(ctx, s))) break;
            } else if ((rc = build_f32c(ctx, t))) {
                break;
            }
        }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_fail(ctx, e, "init sync");
    } while (0);
    if (rc != NBODY_OK) {
        nbody_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return NBODY_OK;
}

int nbody_tune(nbody_ctx *ctx, void *stream) {
    int rc = guard(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = run_tuner(ctx, s))) return rc;
    NB_CUDA(cudaStreamSynchronize(s));
    return NBODY_OK;
}

int nbody_get_tiles(const nbody_ctx *ctx, nbody_tiles *out) {
    if (!ctx || !out) return NBODY_EINVAL;
    *out = ctx->mode == NBODY_F32C ? ctx->tiles : nbody_tiles{0, 0, 0, 0, 0};
    return NBODY_OK;
}

int64_t nbody_kernel_launches(const nbody_ctx *ctx) { return ctx ? ctx->launches : 0; }

int nbody_block_trace(nbody_ctx *ctx, uint64_t *out, int64_t first, int64_t count, void *stream) {
    int rc = guard(ctx);
    if (rc) return rc;
    if (!(ctx->flags & NBODY_FLAG_TRACE) || !ctx->bs.trace)
        return fail(ctx, NBODY_ESTATE, "no trace: NBODY_FLAG_TRACE with NBODY_F32C block steps");
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(cudaStreamSynchronize(s));
    long long blocks = 0;
    NB_CUDA(cudaMemcpy(&blocks, &ctx->bs.sc->blocks, sizeof blocks, cudaMemcpyDeviceToHost));
    if (count < 0 || first < 0 || (count > 0 && !out) || first + count > blocks + 1 ||
        count > NBODY_TRACE_CAP || blocks + 1 - first > NBODY_TRACE_CAP)
        return fail(ctx, NBODY_EINVAL, "trace records out of range");
    for (int64_t k = 0; k < count;) {  // the ring in at most two pieces
        const int64_t at = (first + k) % NBODY_TRACE_CAP;
        const int64_t piece = std::min<int64_t>(count - k, NBODY_TRACE_CAP - at);
        NB_CUDA(cudaMemcpy(out + 2 * k, ctx->bs.trace + 2 * at, (size_t)piece * 2 * sizeof(uint64_t),
                           cudaMemcpyDeviceToHost));
        k += piece;
    }
    return NBODY_OK;
}

int nbody_profile_read(nbody_ctx *ctx, double *ms_total, int64_t *launches, int reset) {
    if (!ctx) return NBODY_EINVAL;
    for (int sl = 0; sl < kProfSlots; ++sl) {
        int rc = prof_drain(ctx, sl);
        if (rc) return rc;
    }
    if (ms_total) *ms_total = ctx->prof_ms;
    if (launches) *launches = ctx->prof_count;
    if (reset) {
        ctx->prof_ms = 0.0;
        ctx->prof_count = 0;
    }
    return NBODY_OK;
}

int nbody_forces(nbody_ctx *ctx, const double *pos, const double *mass, double *acc, double *pot,
                 void *stream) {
    int rc = guard(ctx);
    if (rc) return rc;
    if (ctx->n == 0) return NBODY_OK;
    if ((rc = check_ptr(ctx, pos, "pos", true)) || (rc = check_ptr(ctx, mass, "mass", true)) ||
        (rc = check_ptr(ctx, acc, "acc", true)) || (rc = check_ptr(ctx, pot, "pot", false)))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n3b = 3 * ctx->n * sizeof(double), nb = ctx->n * sizeof(double);
    void *dpos, *dmass, *dacc, *dpot;
    bool spos, smass, sacc, spot;
    if ((rc = resolve(ctx, pos, n3b, ctx->st_pos, true, s, &dpos, &spos)) ||
        (rc = resolve(ctx, mass, nb, ctx->st_mass, true, s, &dmass, &smass)) ||
        (rc = resolve(ctx, acc, n3b, ctx->st_acc, false, s, &dacc, &sacc)) ||
        (rc = resolve(ctx, pot, nb, ctx->st_pot, false, s, &dpot, &spot)))
        return rc;
    Arrays a{(double *)dpos, nullptr, (double *)dacc, (double *)dpot, nullptr, (const double *)dmass};
    const int slot = next_slot(ctx);
    if (slot < -1) return ctx->sticky;
    int k = 0;
    rc = enqueue_forces(ctx, a, 0.0, want_reorder(ctx), slot, false, s, &k);
    ctx->launches += k;
    if (rc) return rc;
    if (slot >= 0) ctx->ev_pending[slot] = true;
    ctx->evals += 1;
    if (sacc) NB_CUDA(cudaMemcpyAsync(acc, dacc, n3b, cudaMemcpyDeviceToHost, s));
    if (spot) NB_CUDA(cudaMemcpyAsync(pot, dpot, nb, cudaMemcpyDeviceToHost, s));
    if (sacc || spot) NB_CUDA(cudaStreamSynchronize(s));
    return check_finite(ctx, (const double *)dacc, (const double *)dpot, s);
}

}  // extern "C"

namespace {

// KDK (kind 0) or Hermite (kind 1, jerk != null) steps, eager or graph-replayed.
int step_common(nbody_ctx *ctx, double *pos, double *vel, const double *mass, double *acc,
                double *jerk, double *pot, double dt, int32_t nsteps, double *diag, void *stream,
                int kind) {
    int rc = guard(ctx);
    if (rc) return rc;
    if (!std::isfinite(dt)) return fail(ctx, NBODY_EINVAL, "dt is not finite");
    if (nsteps < 0) return fail(ctx, NBODY_EINVAL, "nsteps < 0");
    if (ctx->n == 0 || nsteps == 0) return NBODY_OK;
    if ((rc = check_ptr(ctx, pos, "pos", true)) || (rc = check_ptr(ctx, vel, "vel", true)) ||
        (rc = check_ptr(ctx, mass, "mass", true)) || (rc = check_ptr(ctx, acc, "acc", true)) ||
        (rc = check_ptr(ctx, pot, "pot", false)) || (rc = check_ptr(ctx, diag, "diag", false)) ||
        (rc = check_ptr(ctx, jerk, "jerk", kind >= 1)))
        return rc;
    if (kind >= 1 && (rc = ensure_jerk(ctx))) return rc;
    if (kind == 2 && !ctx->bs.started) return fail(ctx, NBODY_EINVAL, "nbody_block_start was not called");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n3b = 3 * ctx->n * sizeof(double), nb = ctx->n * sizeof(double);
    const size_t db = (size_t)nsteps * ctx->ncl * 9 * sizeof(double);
    void *dpos, *dvel, *dmass, *dacc, *dpot, *ddiag, *djerk = nullptr;
    bool spos, svel, smass, sacc, spot, sdiag, sjerk = false;
    if ((rc = resolve(ctx, pos, n3b, ctx->st_pos, true, s, &dpos, &spos)) ||
        (rc = resolve(ctx, vel, n3b, ctx->st_vel, true, s, &dvel, &svel)) ||
        (rc = resolve(ctx, mass, nb, ctx->st_mass, true, s, &dmass, &smass)) ||
        (rc = resolve(ctx, acc, n3b, ctx->st_acc, true, s, &dacc, &sacc)) ||
        (rc = resolve(ctx, pot, nb, ctx->st_pot, true, s, &dpot, &spot)) ||
        (rc = resolve(ctx, diag, db, ctx->st_diag, false, s, &ddiag, &sdiag)) ||
        (rc = resolve(ctx, jerk, n3b, ctx->st_jerk, true, s, &djerk, &sjerk)))
        return rc;
    Arrays a{(double *)dpos, (double *)dvel, (double *)dacc, (double *)dpot, (double *)ddiag,
             (const double *)dmass, (double *)djerk};
    if (a.diag) NB_CUDA(cudaMemsetAsync(ctx->diag_counter, 0, sizeof(int), s));
    const bool use_graph = !(ctx->flags & NBODY_FLAG_NO_GRAPH);
    uint64_t dt_bits;
    memcpy(&dt_bits, &dt, sizeof dt);
    for (int32_t step = 0; step < nsteps; ++step) {
        bool reorder = want_reorder(ctx), fresh = false;
        if (kind == 2) {
            reorder = ctx->bs.reorder_pending;
            fresh = reorder || ctx->bs.fresh_pending;
            ctx->bs.reorder_pending = ctx->bs.fresh_pending = false;
        }
        // graph variants: 0 plain, 1 re-sort; block steps: 1 fresh pack, 2 re-sort + fresh pack
        const int variant = kind == 2 ? (reorder ? 2 : fresh ? 1 : 0) : (reorder ? 1 : 0);
        const int slot = next_slot(ctx);
        if (slot < -1) return ctx->sticky;
        const int multi =
            kind == 2 && use_graph && slot == -1 && !fresh && nsteps - step >= kMultiSteps ? kMultiSteps : 1;
        if (!use_graph) {
            int k = 0;
            rc = kind == 2   ? enqueue_block_step(ctx, a, reorder, fresh, slot, false, s, &k)
                 : kind == 1 ? enqueue_hermite_step(ctx, a, dt, reorder, slot, false, s, &k)
                             : enqueue_step(ctx, a, dt, reorder, slot, false, s, &k);
            ctx->launches += k;
            if (rc) return rc;
        } else {
            GraphEntry *g = nullptr;
            for (auto &e : ctx->graphs)
                if (e.pos == a.pos && e.vel == a.vel && e.mass == a.mass && e.acc == a.acc &&
                    e.pot == a.pot && e.diag == a.diag && e.jerk == a.jerk && e.kind == kind &&
                    e.dt_bits == dt_bits && e.reorder == variant && e.slot == slot &&
                    e.steps == multi)
                    g = &e;
            if (!g) {
                if (ctx->graphs.size() >= 16) drop_graphs(ctx);
                GraphEntry ge{a.pos, a.vel, a.mass, a.acc, a.pot, a.diag, a.jerk, kind, dt_bits,
                              variant, slot, nullptr, 0, multi};
                NB_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
                int k = 0;
                for (int m = 0; m < multi && rc == NBODY_OK; ++m)
                    rc = kind == 2   ? enqueue_block_step(ctx, a, reorder, fresh, slot, true, ctx->cap_stream, &k)
                         : kind == 1 ? enqueue_hermite_step(ctx, a, dt, reorder, slot, true, ctx->cap_stream, &k)
                                     : enqueue_step(ctx, a, dt, reorder, slot, true, ctx->cap_stream, &k);
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
                if (rc) {
                    if (graph) cudaGraphDestroy(graph);
                    return rc;
                }
                if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&ge.exec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
                ge.kernels = k;
                ctx->graphs.push_back(ge);
                g = &ctx->graphs.back();
            }
            NB_CUDA(cudaGraphLaunch(g->exec, s));
            ctx->launches += g->kernels;
        }
        if (slot >= 0) ctx->ev_pending[slot] = true;
        ctx->evals += 1;
        if (use_graph && multi > 1) {
            step += multi - 1;
            ctx->evals += multi - 1;
        }
    }
    if (spos) NB_CUDA(cudaMemcpyAsync(pos, dpos, n3b, cudaMemcpyDeviceToHost, s));
    if (svel) NB_CUDA(cudaMemcpyAsync(vel, dvel, n3b, cudaMemcpyDeviceToHost, s));
    if (sacc) NB_CUDA(cudaMemcpyAsync(acc, dacc, n3b, cudaMemcpyDeviceToHost, s));
    if (spot) NB_CUDA(cudaMemcpyAsync(pot, dpot, nb, cudaMemcpyDeviceToHost, s));
    if (sdiag) NB_CUDA(cudaMemcpyAsync(diag, ddiag, db, cudaMemcpyDeviceToHost, s));
    if (sjerk) NB_CUDA(cudaMemcpyAsync(jerk, djerk, n3b, cudaMemcpyDeviceToHost, s));
    if (spos || svel || sacc || spot || sdiag || sjerk) NB_CUDA(cudaStreamSynchronize(s));
    return check_finite(ctx, (const double *)dacc, (const double *)dpot, s);
}

}  // namespace

extern "C" {

int nbody_step(nbody_ctx *ctx, double *pos, double *vel, const double *mass, double *acc,
               double *pot, double dt, int32_t nsteps, double *diag, void *stream) {
    return step_common(ctx, pos, vel, mass, acc, nullptr, pot, dt, nsteps, diag, stream, 0);
}

int nbody_step_hermite(nbody_ctx *ctx, double *pos, double *vel, const double *mass, double *acc,
                       double *jerk, double *pot, double dt, int32_t nsteps, double *diag,
                       void *stream) {
    return step_common(ctx, pos, vel, mass, acc, jerk, pot, dt, nsteps, diag, stream, 1);
}

int nbody_forces_jerk(nbody_ctx *ctx, const double *pos, const double *vel, const double *mass,
                      double *acc, double *jerk, double *pot, void *stream) {
    int rc = guard(ctx);
    if (rc) return rc;
    if (ctx->n == 0) return NBODY_OK;
    if ((rc = check_ptr(ctx, pos, "pos", true)) || (rc = check_ptr(ctx, vel, "vel", true)) ||
        (rc = check_ptr(ctx, mass, "mass", true)) || (rc = check_ptr(ctx, acc, "acc", true)) ||
        (rc = check_ptr(ctx, jerk, "jerk", true)) || (rc = check_ptr(ctx, pot, "pot", false)))
        return rc;
    if ((rc = ensure_jerk(ctx))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n3b = 3 * ctx->n * sizeof(double), nb = ctx->n * sizeof(double);
    void *dpos, *dvel, *dmass, *dacc, *djerk, *dpot;
    bool spos, svel, smass, sacc, sjerk, spot;
    if ((rc = resolve(ctx, pos, n3b, ctx->st_pos, true, s, &dpos, &spos)) ||
        (rc = resolve(ctx, vel, n3b, ctx->st_vel, true, s, &dvel, &svel)) ||
        (rc = resolve(ctx, mass, nb, ctx->st_mass, true, s, &dmass, &smass)) ||
        (rc = resolve(ctx, acc, n3b, ctx->st_acc, false, s, &dacc, &sacc)) ||
        (rc = resolve(ctx, jerk, n3b, ctx->st_jerk, false, s, &djerk, &sjerk)) ||
        (rc = resolve(ctx, pot, nb, ctx->st_pot, false, s, &dpot, &spot)))
        return rc;
    const int slot = next_slot(ctx);
    if (slot < -1) return ctx->sticky;
    int k = 0;
    rc = enqueue_forces_jerk(ctx, (const double *)dpos, (const double *)dvel, (const double *)dmass,
                             (double *)dacc, (double *)djerk, (double *)dpot, want_reorder(ctx), slot,
                             false, s, &k);
    ctx->launches += k;
    if (rc) return rc;
    if (slot >= 0) ctx->ev_pending[slot] = true;
    ctx->evals += 1;
    if (sacc) NB_CUDA(cudaMemcpyAsync(acc, dacc, n3b, cudaMemcpyDeviceToHost, s));
    if (sjerk) NB_CUDA(cudaMemcpyAsync(jerk, djerk, n3b, cudaMemcpyDeviceToHost, s));
    if (spot) NB_CUDA(cudaMemcpyAsync(pot, dpot, nb, cudaMemcpyDeviceToHost, s));
    if (sacc || sjerk || spot) NB_CUDA(cudaStreamSynchronize(s));
    return check_finite(ctx, (const double *)dacc, (const double *)dpot, s);
}

static bool pow2(double x) { return x > 0.0 && std::isfinite(x) && std::exp2(std::round(std::log2(x))) == x; }

int nbody_block_start(nbody_ctx *ctx, const double *pos, const double *vel, const double *mass,
                      double *acc, double *jerk, double *pot, double dt_max, double dt_min,
                      double eta, double eta_s, void *stream) {
    int rc = guard(ctx);
    if (rc) return rc;
    if (!pow2(dt_max) || !pow2(dt_min) || dt_min > dt_max || !(eta > 0.0) || !(eta_s > 0.0) ||
        !std::isfinite(eta) || !std::isfinite(eta_s))
        return fail(ctx, NBODY_EINVAL, "block steps: dt_max, dt_min must be powers of two, eta > 0");
    if (dt_max / dt_min > 0x1p40)
        return fail(ctx, NBODY_EINVAL, "block steps: dt_max / dt_min must be at most 2^40");
    if (ctx->mode == NBODY_F32C && dt_min < 0x1p-126)
        return fail(ctx, NBODY_EINVAL, "F32C block steps: dt_min must be at least 2^-126 (a normal float)");
    if (ctx->n == 0) return NBODY_OK;
    for (const void *q : {(const void *)pos, (const void *)vel, (const void *)mass, (const void *)acc,
                          (const void *)jerk})
        if (!q || !is_device_ptr(q)) return fail(ctx, NBODY_EINVAL, "block steps need device arrays");
    if (pot && !is_device_ptr(pot)) return fail(ctx, NBODY_EINVAL, "block steps need device arrays");
    if (!ctx->jp.built && (rc = build_jerk(ctx, default_jerk_tiles(ctx, true)))) return rc;
    if ((rc = alloc_block(ctx))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = nbody_forces_jerk(ctx, pos, vel, mass, acc, jerk, pot, stream))) return rc;
    BlockState &b = ctx->bs;
    b.dt_max = dt_max;
    b.dt_min = dt_min;
    b.eta = eta;
    NB_CUDA(launch_block_init(ctx->n, acc, jerk, dt_max, dt_min, eta_s, b.t, b.dt, b.tq, s));
    NB_CUDA(cudaMemsetAsync(b.sc, 0, sizeof(BlockScalars), s));
    // level counts and the first t_next (later steps set the next one themselves)
    NB_CUDA(launch_block_levels(ctx->n, b.dt, dt_max, dt_min, ctx->chunks, ctx->n_chunks, b.tq, b.part,
                                b.sc, s));
    ctx->launches += 3;
    NB_CUDA(cudaStreamSynchronize(s));
    b.reorder_epoch = 0;
    b.reorder_pending = false;
    b.fresh_pending = true;
    b.started = true;
    return NBODY_OK;
}

int nbody_block_advance(nbody_ctx *ctx, double *pos, double *vel, const double *mass, double *acc,
                        double *jerk, double *pot, double t_end, int64_t *blocks, int64_t *evals,
                        void *stream) {
    int rc = guard(ctx);
    if (rc) return rc;
    if (ctx->n == 0) return NBODY_OK;
    BlockState &b = ctx->bs;
    if (!b.started) return fail(ctx, NBODY_EINVAL, "nbody_block_start was not called");
    if (!std::isfinite(t_end) || t_end < 0.0 || std::fmod(t_end, b.dt_max) != 0.0)
        return fail(ctx, NBODY_EINVAL, "t_end must be a non-negative multiple of dt_max");
    if (t_end / b.dt_min > 0x1p60)
        return fail(ctx, NBODY_EINVAL, "t_end / dt_min must be at most 2^60 (times are counted in dt_min)");
    for (const void *q : {(const void *)pos, (const void *)vel, (const void *)mass, (const void *)acc,
                          (const void *)jerk})
        if (!q || !is_device_ptr(q)) return fail(ctx, NBODY_EINVAL, "block steps need device arrays");
    if (pot && !is_device_ptr(pot)) return fail(ctx, NBODY_EINVAL, "block steps need device arrays");
    cudaStream_t s = (cudaStream_t)stream;
    b.fresh_pending = true;  // the rows are the caller's: take them as they are now
    struct {
        double t;
        long long q;
    } end{t_end, (long long)(t_end / b.dt_min)};  // exact: t_end a multiple of dt_max
    static_assert(offsetof(BlockScalars, t_end_q) == offsetof(BlockScalars, t_end) + sizeof(double),
                  "t_end, t_end_q adjacent");
    NB_CUDA(cudaMemcpyAsync(&b.sc->t_end, &end, sizeof end, cudaMemcpyHostToDevice, s));
    BlockScalars h{};
    NB_CUDA(cudaMemcpyAsync(&h, b.sc, sizeof h, cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    const double t0 = h.t_next;
    const long long blocks0 = h.blocks;
    int batch = 16;
    for (;;) {
        // steps past t_end find no active particle and change nothing, so a
        // batch may overshoot; its size follows the block-step rate so far
        // (about half the steps still expected, 16..256), which keeps the
        // host round trips few and the wasted steps bounded
        if ((rc = step_common(ctx, pos, vel, mass, acc, jerk, pot, 0.0, batch, nullptr, stream, 2))) return rc;
        NB_CUDA(cudaMemcpyAsync(&h, b.sc, sizeof h, cudaMemcpyDeviceToHost, s));
        NB_CUDA(cudaStreamSynchronize(s));
        const double next = (double)block_next_time_q(h.t_next_q, h.n_active, h.level, b.dt_max, b.dt_min) * b.dt_min;
        if (!(next <= t_end)) break;
        const double done = h.t_next - t0;
        if (done > 0.0) {
            const double rate = (double)(h.blocks - blocks0) / done;
            const double left = rate * (t_end - h.t_next);
            batch = (int)std::min(256.0, std::max(16.0, 0.5 * left));
        }
        if (ctx->mode == NBODY_F32C && ctx->reorder_every > 0) {
            const int64_t epoch = (int64_t)std::floor(h.t_next / (ctx->reorder_every * b.dt_max));
            if (epoch > b.reorder_epoch) {
                b.reorder_epoch = epoch;
                b.reorder_pending = true;
            }
        }
    }
    if (b.trace) NB_CUDA(launch_block_trace_end(b.sc, b.trace, NBODY_TRACE_CAP, s));
    if (blocks) *blocks = h.blocks;
    if (evals) *evals = h.evals;
    return NBODY_OK;
}

int nbody_block_state(nbody_ctx *ctx, double *t_host, double *dt_host, void *stream) {
    int rc = guard(ctx);
    if (rc) return rc;
    if (ctx->n == 0) return NBODY_OK;
    if (!ctx->bs.started) return fail(ctx, NBODY_EINVAL, "nbody_block_start was not called");
    cudaStream_t s = (cudaStream_t)stream;
    if (t_host) NB_CUDA(cudaMemcpyAsync(t_host, ctx->bs.t, ctx->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (dt_host) NB_CUDA(cudaMemcpyAsync(dt_host, ctx->bs.dt, ctx->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    return NBODY_OK;
}

int nbody_get_jerk_tiles(const nbody_ctx *ctx, nbody_tiles *out) {
    if (!ctx || !out) return NBODY_EINVAL;
    *out = ctx->mode == NBODY_F32C && ctx->jp.built ? ctx->jp.tiles : nbody_tiles{0, 0, 0, 0, 0};
    return NBODY_OK;
}

int nbody_set_jerk_tiles(nbody_ctx *ctx, const nbody_tiles *t) {
    int rc = guard(ctx);
    if (rc) return rc;
    if (!t) return fail(ctx, NBODY_EINVAL, "tiles is NULL");
    if (ctx->mode != NBODY_F32C) return NBODY_OK;
    return build_jerk(ctx, *t);
}

int nbody_energy(nbody_ctx *ctx, const double *pos, const double *vel, const double *mass,
                 const double *pot, double *out_host, void *stream) {
    int rc = guard(ctx);
    if (rc) return rc;
    if ((rc = check_ptr(ctx, out_host, "out_host", true))) return rc;
    if (ctx->n == 0) {
        for (int k = 0; k < 9 * ctx->ncl; ++k) out_host[k] = 0.0;
        return NBODY_OK;
    }
    if ((rc = check_ptr(ctx, pos, "pos", true)) || (rc = check_ptr(ctx, vel, "vel", true)) ||
        (rc = check_ptr(ctx, mass, "mass", true)) || (rc = check_ptr(ctx, pot, "pot", false)))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n3b = 3 * ctx->n * sizeof(double), nb = ctx->n * sizeof(double);
    void *dpos, *dvel, *dmass, *dpot;
    bool a1, a2, a3, a4;
    if ((rc = resolve(ctx, pos, n3b, ctx->st_pos, true, s, &dpos, &a1)) ||
        (rc = resolve(ctx, vel, n3b, ctx->st_vel, true, s, &dvel, &a2)) ||
        (rc = resolve(ctx, mass, nb, ctx->st_mass, true, s, &dmass, &a3)) ||
        (rc = resolve(ctx, pot, nb, ctx->st_pot, true, s, &dpot, &a4)))
        return rc;
    NB_CUDA(launch_energy((const double *)dpos, (const double *)dvel, (const double *)dmass,
                          (const double *)dpot, ctx->n, ctx->chunks, ctx->n_chunks, ctx->chunk_first,
                          ctx->ncl, ctx->epart, ctx->edev, nullptr, s));
    ctx->launches += ctx->n_chunks > 0 ? 2 : 1;
    NB_CUDA(cudaMemcpyAsync(out_host, ctx->edev, (size_t)ctx->ncl * 9 * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    return NBODY_OK;
}

}  // extern "C"
