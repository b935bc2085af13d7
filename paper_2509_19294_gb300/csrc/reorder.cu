// reorder.cu -- Morton-curve regrouping of particles into compact tiles.
//
// The F32C kernel measures every particle from its tile's FP64 centre in FP32,
// so the error of a close pair's separation scales with the tile's spatial
// extent.  Sorting each cluster's particles along a Morton (Z-order) curve of
// its own bounding box makes tiles spatially compact.  This only changes which
// particles share a tile (and hence rounding), never the quantity computed.
//
// Steps: per-cluster bounding box (two-stage min/max, exact), 30-bit Morton key
// (10 bits per axis) with the cluster id in the high word, a bitonic sort of
// (key, row) pairs (all pairs distinct, so the order is unique), then
// perm[slot] = row for every real slot.
//
// When every cluster has at most kSmemSortMax particles (ensembles of small
// systems) one CTA per cluster does all four steps in shared memory, sorting
// (key << 32 | local index); that gives the same order as the global sort.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "nbody_internal.h"

namespace nbody {

namespace {

constexpr int kSortChunk = 2048;          // elements sorted per CTA in shared memory
constexpr int kSortThreads = kSortChunk / 2;
constexpr int kBoxThreads = 256;

__global__ void __launch_bounds__(kBoxThreads)
    bbox_chunk_kernel(const double *__restrict__ pos, int64_t n, const Chunk *__restrict__ chunks,
                      double *__restrict__ part) {
    __shared__ double red[kBoxThreads / 32][6];
    const Chunk ch = chunks[blockIdx.x];
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = ch.begin + threadIdx.x; i < ch.end; i += kBoxThreads) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = pos[d * n + i];
            v[d] = fmin(v[d], x);
            v[3 + d] = fmax(v[3 + d], x);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            v[d] = fmin(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
            v[3 + d] = fmax(v[3 + d], __shfl_xor_sync(0xffffffffu, v[3 + d], o));
        }
    if (threadIdx.x % 32 == 0)
#pragma unroll
        for (int d = 0; d < 6; ++d) red[threadIdx.x / 32][d] = v[d];
    __syncthreads();
    if (threadIdx.x < 6) {
        const int d = threadIdx.x;
        double r = red[0][d];
        for (int w = 1; w < kBoxThreads / 32; ++w) r = d < 3 ? fmin(r, red[w][d]) : fmax(r, red[w][d]);
        part[6 * blockIdx.x + d] = r;
    }
}

__global__ void bbox_cluster_kernel(const double *__restrict__ part,
                                    const int32_t *__restrict__ chunk_first, int ncl,
                                    double *__restrict__ bbox) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncl; c += gridDim.x * blockDim.x) {
        double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int k = chunk_first[c]; k < chunk_first[c + 1]; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                v[d] = fmin(v[d], part[6 * k + d]);
                v[3 + d] = fmax(v[3 + d], part[6 * k + 3 + d]);
            }
#pragma unroll
        for (int d = 0; d < 6; ++d) bbox[6 * c + d] = v[d];
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    // insert two zero bits between each of the low 10 bits
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t cell10(double x, double lo, double hi) {
    const double w = hi - lo;
    if (!(w > 0.0)) return 0u;
    double q = (x - lo) / w * 1024.0;
    q = fmin(fmax(q, 0.0), 1023.0);
    return (uint32_t)q;
}

__global__ void morton_kernel(const double *__restrict__ pos, int64_t n,
                              const Chunk *__restrict__ chunks, const double *__restrict__ bbox,
                              unsigned long long *__restrict__ keys, uint32_t *__restrict__ vals) {
    const Chunk ch = chunks[blockIdx.x];
    const double *b = bbox + 6 * ch.cluster;
    for (int64_t i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) {
        const uint32_t m = (spread10(cell10(pos[i], b[0], b[3])) << 2) |
                           (spread10(cell10(pos[n + i], b[1], b[4])) << 1) |
                           spread10(cell10(pos[2 * n + i], b[2], b[5]));
        keys[i] = ((unsigned long long)(uint32_t)ch.cluster << 32) | m;
        vals[i] = (uint32_t)i;
    }
}

__global__ void sort_pad_kernel(int64_t n, int64_t sort_n, unsigned long long *keys,
                                uint32_t *vals) {
    for (int64_t q = n + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < sort_n;
         q += (int64_t)gridDim.x * blockDim.x) {
        keys[q] = ~0ull;
        vals[q] = 0xffffffffu;
    }
}

__device__ __forceinline__ bool pair_greater(unsigned long long ka, uint32_t va,
                                             unsigned long long kb, uint32_t vb) {
    return ka > kb || (ka == kb && va > vb);
}

// Bitonic stages inside one CTA's chunk.  full: all stages k = 2..chunk;
// otherwise the j < chunk steps of stage k.
__global__ void __launch_bounds__(kSortThreads)
    bitonic_smem_kernel(unsigned long long *keys, uint32_t *vals, int64_t chunk, int full,
                        int64_t kstage) {
    __shared__ unsigned long long sk[kSortChunk];
    __shared__ uint32_t sv[kSortChunk];
    const int64_t base = (int64_t)blockIdx.x * chunk;
    for (int q = threadIdx.x; q < chunk; q += blockDim.x) {
        sk[q] = keys[base + q];
        sv[q] = vals[base + q];
    }
    __syncthreads();
    const int64_t k_lo = full ? 2 : kstage, k_hi = full ? chunk : kstage;
    for (int64_t k = k_lo; k <= k_hi; k <<= 1) {
        for (int64_t j = (full ? k : chunk) >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < chunk / 2; t += blockDim.x) {
                const int i = 2 * (int)j * (t / (int)j) + (t % (int)j);
                const int l = i + (int)j;
                const bool up = ((base + i) & k) == 0;
                const bool gt = pair_greater(sk[i], sv[i], sk[l], sv[l]);
                if (gt == up) {
                    const unsigned long long tk = sk[i];
                    sk[i] = sk[l];
                    sk[l] = tk;
                    const uint32_t tv = sv[i];
                    sv[i] = sv[l];
                    sv[l] = tv;
                }
            }
            __syncthreads();
        }
    }
    for (int q = threadIdx.x; q < chunk; q += blockDim.x) {
        keys[base + q] = sk[q];
        vals[base + q] = sv[q];
    }
}

// One compare-exchange step (stage k, distance j >= chunk) over the whole array.
__global__ void bitonic_global_kernel(unsigned long long *keys, uint32_t *vals, int64_t half,
                                      int64_t k, int64_t j) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < half;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = 2 * j * (t / j) + (t % j);
        const int64_t l = i + j;
        const bool up = (i & k) == 0;
        const unsigned long long ki = keys[i], kl = keys[l];
        const uint32_t vi = vals[i], vl = vals[l];
        if (pair_greater(ki, vi, kl, vl) == up) {
            keys[i] = kl;
            keys[l] = ki;
            vals[i] = vl;
            vals[l] = vi;
        }
    }
}

__global__ void perm_kernel(int64_t n, const unsigned long long *__restrict__ keys,
                            const uint32_t *__restrict__ vals, const ClusterDev *__restrict__ cl,
                            int32_t *__restrict__ perm) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(keys[q] >> 32);
        const ClusterDev d = cl[c];
        perm[d.slot_begin + (q - d.user_begin)] = (int32_t)vals[q];
    }
}

constexpr int kSmemSortThreads = 1024;

__global__ void __launch_bounds__(kSmemSortThreads)
    cluster_reorder_kernel(const double *__restrict__ pos, int64_t n,
                           const ClusterDev *__restrict__ cl, int32_t *__restrict__ perm,
                           int pow2) {
    extern __shared__ unsigned long long sk[];  // pow2 keys
    __shared__ double red[kSmemSortThreads / 32][6];
    __shared__ double box[6];
    const ClusterDev d = cl[blockIdx.x];
    if (d.n == 0) return;
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int k = threadIdx.x; k < d.n; k += blockDim.x) {
        const int64_t i = d.user_begin + k;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double x = pos[q * n + i];
            v[q] = fmin(v[q], x);
            v[3 + q] = fmax(v[3 + q], x);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            v[q] = fmin(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
            v[3 + q] = fmax(v[3 + q], __shfl_xor_sync(0xffffffffu, v[3 + q], o));
        }
    if (threadIdx.x % 32 == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q) red[threadIdx.x / 32][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 6) {
        const int q = threadIdx.x;
        double r = red[0][q];
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) r = q < 3 ? fmin(r, red[w][q]) : fmax(r, red[w][q]);
        box[q] = r;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < pow2; k += blockDim.x) {
        unsigned long long key = ~0ull;
        if (k < d.n) {
            const int64_t i = d.user_begin + k;
            const uint32_t m = (spread10(cell10(pos[i], box[0], box[3])) << 2) |
                               (spread10(cell10(pos[n + i], box[1], box[4])) << 1) |
                               spread10(cell10(pos[2 * n + i], box[2], box[5]));
            key = ((unsigned long long)m << 32) | (uint32_t)k;
        }
        sk[k] = key;
    }
    __syncthreads();
    for (int kk = 2; kk <= pow2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < pow2 / 2; t += blockDim.x) {
                const int i = 2 * j * (t / j) + (t % j);
                const int l = i + j;
                const bool up = (i & kk) == 0;
                const unsigned long long a = sk[i], b = sk[l];
                if ((a > b) == up) {
                    sk[i] = b;
                    sk[l] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < d.n; k += blockDim.x)
        perm[d.slot_begin + k] = (int32_t)(d.user_begin + (uint32_t)(sk[k] & 0xffffffffu));
}

int grid_cap(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

bool reorder_in_smem(int64_t max_cluster) { return max_cluster <= kSmemSortMax; }

cudaError_t launch_reorder(const double *pos, int64_t n, const Chunk *chunks, int n_chunks,
                           const int32_t *chunk_first, int ncl, const ClusterDev *cl,
                           double *part, double *bbox, unsigned long long *keys, uint32_t *vals,
                           int64_t sort_n, int64_t max_cluster, int32_t *perm, cudaStream_t s,
                           int *launches) {
    if (n <= 0 || n_chunks <= 0) return cudaSuccess;
    cudaError_t e;
#define NB_CHECK()                             \
    do {                                       \
        e = cudaGetLastError();                \
        if (e != cudaSuccess) return e;        \
        if (launches) ++*launches;             \
    } while (0)
    if (reorder_in_smem(max_cluster)) {
        int pow2 = 1;
        while (pow2 < max_cluster) pow2 <<= 1;
        const size_t smem = sizeof(unsigned long long) * pow2;
        e = cudaFuncSetAttribute(cluster_reorder_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        const int threads = pow2 / 2 < kSmemSortThreads ? (pow2 / 2 < 32 ? 32 : pow2 / 2)
                                                         : kSmemSortThreads;
        cluster_reorder_kernel<<<ncl, threads, smem, s>>>(pos, n, cl, perm, pow2);
        NB_CHECK();
        return cudaSuccess;
    }
    bbox_chunk_kernel<<<n_chunks, kBoxThreads, 0, s>>>(pos, n, chunks, part);
    NB_CHECK();
    bbox_cluster_kernel<<<grid_cap(ncl, 128), 128, 0, s>>>(part, chunk_first, ncl, bbox);
    NB_CHECK();
    morton_kernel<<<n_chunks, 256, 0, s>>>(pos, n, chunks, bbox, keys, vals);
    NB_CHECK();
    if (sort_n > n) {
        sort_pad_kernel<<<grid_cap(sort_n - n, 256), 256, 0, s>>>(n, sort_n, keys, vals);
        NB_CHECK();
    }
    const int64_t chunk = sort_n < kSortChunk ? sort_n : kSortChunk;
    const int nblk = (int)(sort_n / chunk);
    bitonic_smem_kernel<<<nblk, kSortThreads, 0, s>>>(keys, vals, chunk, 1, 0);
    NB_CHECK();
    for (int64_t k = 2 * chunk; k <= sort_n; k <<= 1) {
        for (int64_t j = k >> 1; j >= chunk; j >>= 1) {
            bitonic_global_kernel<<<grid_cap(sort_n / 2, 256), 256, 0, s>>>(keys, vals, sort_n / 2,
                                                                              k, j);
            NB_CHECK();
        }
        bitonic_smem_kernel<<<nblk, kSortThreads, 0, s>>>(keys, vals, chunk, 0, k);
        NB_CHECK();
    }
    perm_kernel<<<grid_cap(n, 256), 256, 0, s>>>(n, keys, vals, cl, perm);
    NB_CHECK();
#undef NB_CHECK
    return cudaSuccess;
}

}  // namespace nbody
