// noalloc.cu -- nbody_forces_noalloc: the FP32-compensated force evaluation of
// one system without any memory allocation.
//
// Who needs it: callers that must not allocate device memory at the time they
// compute forces -- for example code that runs inside a memory pool or arena
// it does not own, real-time loops whose allocation latency is not allowed, or
// plug-ins hosted by a process that has reserved the whole GPU memory for
// itself.  nbody_init allocates the scratch of a context with cudaMalloc, so
// such callers cannot use it.  This entry point instead keeps its scratch in a
// fixed array compiled into the library (g_scratch below): every GPU that loads
// libnbody.so holds it until the process exits, whether or not it is used.
//
// What it computes: exactly what nbody_forces computes for a single system in
// NBODY_F32C mode (no reordering), with a fixed tile shape (128 threads, 2
// i-particles per thread, 256 j-particles per shared tile) and a split count
// chosen from n.  It reuses the library's pack and force kernels unchanged; the
// only new device code is the set-up kernel that writes the work queue, the
// identity permutation and the cluster record into the scratch and zeroes the
// queue counters.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "nbody.h"
#include "nbody_internal.h"

using namespace nbody;

namespace {

constexpr int kBlock = 128, kP = 2, kTJ = 256, kMinB = 4;
constexpr int kTC = kBlock * kP;
constexpr int64_t kMaxN = NBODY_NOALLOC_MAX_N;
constexpr int kMaxTiles = (int)((kMaxN + kTC - 1) / kTC);
constexpr int kMaxSplit = 8;
// Most work items the split may create: the scratch holds this many split
// partial slots (4 resident CTAs x 152 SMs of a GB300).  Per call the split
// aims at min(kSplitBudget, resident CTAs of this GPU) items.
constexpr int kSplitBudget = 608;

// Byte layout of the scratch (every region 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffPx = 0;
constexpr size_t kOffPy = kOffPx + align256(sizeof(float) * kMaxTiles * kTC);
constexpr size_t kOffPz = kOffPy + align256(sizeof(float) * kMaxTiles * kTC);
constexpr size_t kOffPm = kOffPz + align256(sizeof(float) * kMaxTiles * kTC);
constexpr size_t kOffPerm = kOffPm + align256(sizeof(float) * kMaxTiles * kTC);
constexpr size_t kOffChl = kOffPerm + align256(sizeof(int32_t) * kMaxTiles * kTC);
constexpr size_t kOffTileCl = kOffChl + align256(sizeof(float4) * 2 * kMaxTiles);
constexpr size_t kOffCounters = kOffTileCl + align256(sizeof(int32_t) * kMaxTiles);
constexpr size_t kOffCl = kOffCounters + align256(sizeof(int) * (kMaxTiles + 1));
constexpr size_t kMaxItems = kSplitBudget > kMaxTiles ? kSplitBudget : kMaxTiles;
constexpr size_t kOffItems = kOffCl + align256(sizeof(ClusterDev));
// partial slots: split > 1 only while n_tiles * split <= kSplitBudget
constexpr size_t kOffPartial = kOffItems + align256(sizeof(Item) * kMaxItems);
constexpr size_t kBytes = kOffPartial + sizeof(double) * 4 * kTC * kSplitBudget;
static_assert(kBytes == NBODY_NOALLOC_SCRATCH_BYTES, "nbody.h states the scratch size");

// The scratch.  In host code g_scratch names a host-side shadow, not the device
// array: its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

std::mutex g_mutex;
constexpr int kMaxDevices = 64;
unsigned char *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Per call: cluster record, identity permutation (pads -1), work queue, and
// zeroed queue head / split tickets.
__global__ void noalloc_setup_kernel(unsigned char *base, int n, int n_tiles, int split,
                                     float eps2f, double eps2) {
    ClusterDev *cl = reinterpret_cast<ClusterDev *>(base + kOffCl);
    int32_t *perm = reinterpret_cast<int32_t *>(base + kOffPerm);
    int32_t *tile_cl = reinterpret_cast<int32_t *>(base + kOffTileCl);
    int *counters = reinterpret_cast<int *>(base + kOffCounters);
    Item *items = reinterpret_cast<Item *>(base + kOffItems);
    const int n_jt = (n + kTJ - 1) / kTJ;
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        ClusterDev d{};
        d.user_begin = 0;
        d.n = n;
        d.slot_begin = 0;
        d.n_jt = n_jt;
        d.eps2f = eps2f;
        d.eps2 = eps2;
        *cl = d;
    }
    for (int s = tid; s < n_tiles * kTC; s += stride) perm[s] = s < n ? s : -1;
    for (int t = tid; t < n_tiles; t += stride) tile_cl[t] = 0;
    for (int t = tid; t <= n_tiles; t += stride) counters[t] = 0;
    for (int k = tid; k < n_tiles * split; k += stride) {
        Item it{};
        it.tile = k / split;
        it.cluster = 0;
        it.split = k % split;
        it.nsplit = split;
        it.jt0 = (int)((int64_t)it.split * n_jt / split);
        it.jt1 = (int)((int64_t)(it.split + 1) * n_jt / split);
        it.pbase = split > 1 ? it.tile * split : 0;
        items[k] = it;
    }
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int nbody_forces_noalloc(int64_t n, const double *pos, const double *mass, double eps,
                                    double G, double *acc, double *pot, void *stream) {
    using std::isfinite;
    if (n < 0 || !isfinite(eps) || eps < 0.0 || !isfinite(G)) return NBODY_EINVAL;
    if (n > kMaxN) return NBODY_ETOOBIG;
    if (n == 0) return NBODY_OK;
    if (!pos || !mass || !acc) return NBODY_EINVAL;
    if (!on_device(pos) || !on_device(mass) || !on_device(acc) || (pot && !on_device(pot)))
        return NBODY_EINVAL;
    cudaGetLastError();  // an error left pending by earlier, unrelated work is not ours
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return NBODY_ECUDA;
    }
    unsigned char *base = nullptr;
    int sms = 0;
    {
        // set-up, once per device and with that device current
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return NBODY_ECUDA;
            }
            int s = 0;
            if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return NBODY_ECUDA;
            }
            g_addr[dev] = static_cast<unsigned char *>(ptr);
            g_sms[dev] = s;
        }
        base = g_addr[dev];
        sms = g_sms[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const float eps2f = (float)(eps * eps);
    const bool eps_zero = eps2f == 0.0f;
    const int n_tiles = (int)((n + kTC - 1) / kTC);
    const int n_jt = (int)((n + kTJ - 1) / kTJ);
    const int occ = f32c_occupancy(kBlock, kP, kTJ, kMinB, eps_zero);
    if (occ <= 0) return NBODY_EUNSUPPORTED;
    const int budget = occ * sms < kSplitBudget ? occ * sms : kSplitBudget;
    int split = budget / n_tiles;
    if (split > kMaxSplit) split = kMaxSplit;
    if (split > n_jt) split = n_jt;
    if (split < 1) split = 1;

    noalloc_setup_kernel<<<64, 256, 0, s>>>(base, (int)n, n_tiles, split, eps2f, eps * eps);
    if (cudaGetLastError() != cudaSuccess) {
        cudaGetLastError();
        return NBODY_ECUDA;
    }

    PackParams pp{};
    pp.pos = pos;
    pp.mass = mass;
    pp.perm = reinterpret_cast<const int32_t *>(base + kOffPerm);
    pp.cl = reinterpret_cast<const ClusterDev *>(base + kOffCl);
    pp.tile_cluster = reinterpret_cast<const int32_t *>(base + kOffTileCl);
    pp.tc = kTC;
    pp.n = n;
    pp.px = reinterpret_cast<float *>(base + kOffPx);
    pp.py = reinterpret_cast<float *>(base + kOffPy);
    pp.pz = reinterpret_cast<float *>(base + kOffPz);
    pp.pm = reinterpret_cast<float *>(base + kOffPm);
    pp.chl = reinterpret_cast<float4 *>(base + kOffChl);
    if (launch_pack(n_tiles, pp, s) != cudaSuccess) {
        cudaGetLastError();
        return NBODY_ECUDA;
    }

    F32CParams fp{};
    fp.px = pp.px;
    fp.py = pp.py;
    fp.pz = pp.pz;
    fp.pm = pp.pm;
    fp.chl = pp.chl;
    fp.perm = pp.perm;
    fp.cl = pp.cl;
    fp.items = reinterpret_cast<const Item *>(base + kOffItems);
    fp.n_items = n_tiles * split;
    fp.tc = kTC;
    fp.counters = reinterpret_cast<int *>(base + kOffCounters);
    fp.partial = reinterpret_cast<double *>(base + kOffPartial);
    fp.acc = acc;
    fp.pot = pot;
    fp.vel = nullptr;
    fp.n = n;
    fp.G = G;
    fp.half_dt = 0.0;
    int grid = occ * sms;
    if (grid > fp.n_items) grid = fp.n_items;
    if (launch_f32c(kBlock, kP, kTJ, kMinB, eps_zero, grid, fp, s) != cudaSuccess) {
        cudaGetLastError();
        return NBODY_ECUDA;
    }
    return NBODY_OK;
}
