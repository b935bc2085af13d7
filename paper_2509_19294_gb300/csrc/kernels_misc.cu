// kernels_misc.cu -- pack, leapfrog, diagnostics and finiteness kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "nbody_internal.h"

namespace nbody {

namespace {

constexpr int kPackWarps = 8;

// Deterministic block sum of NV doubles (fixed shuffle tree, then warps in order).
template <int NT, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*scratch)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += scratch[w][k];
            scratch[0][k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = scratch[0][k];
}

// One warp per centre tile: centre = FP64 mean of the tile's real particles
// (fixed-order shuffle tree, so bitwise reproducible), FP32 offsets from it,
// FP32 masses; pad slots get mass 0 and a far offset.  The centre is stored as
// a float pair hi + lo for the force kernel.  No block barriers: a CTA of
// kPackWarps warps packs kPackWarps independent tiles.
__global__ void __launch_bounds__(kPackWarps * 32) pack_kernel(const PackParams p, int n_tiles) {
    const int lane = threadIdx.x % 32;
    const int t = blockIdx.x * kPackWarps + threadIdx.x / 32;
    if (t >= n_tiles) return;  // warp-uniform
    const ClusterDev cl = p.cl[p.tile_cluster[t]];
    const int base = t * p.tc;
    const int per = p.tc / 32;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int r = 0; r < per; ++r) {
        const int slot = base + lane + 32 * r;
        if (slot - cl.slot_begin < cl.n) {
            const int64_t u = p.perm[slot];
            s[0] += p.pos[u];
            s[1] += p.pos[p.n + u];
            s[2] += p.pos[2 * p.n + u];
            s[3] += 1.0;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    const double cnt = s[3] > 0.0 ? s[3] : 1.0;
    const double cx = s[0] / cnt, cy = s[1] / cnt, cz = s[2] / cnt;
#pragma unroll 4
    for (int r = 0; r < per; ++r) {
        const int slot = base + lane + 32 * r;
        if (slot - cl.slot_begin < cl.n) {
            const int64_t u = p.perm[slot];
            p.px[slot] = (float)(p.pos[u] - cx);
            p.py[slot] = (float)(p.pos[p.n + u] - cy);
            p.pz[slot] = (float)(p.pos[2 * p.n + u] - cz);
            p.pm[slot] = (float)p.mass[u];
        } else {
            p.px[slot] = kPadOffset;
            p.py[slot] = kPadOffset;
            p.pz[slot] = kPadOffset;
            p.pm[slot] = 0.0f;
        }
    }
    if (lane == 0) {
        const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
        p.chl[2 * t + 0] = make_float4(hx, hy, hz, 0.0f);
        p.chl[2 * t + 1] = make_float4((float)(cx - hx), (float)(cy - hy), (float)(cz - hz), 0.0f);
    }
}

// Velocity half of the jerk path's packing (one warp per tile, as pack_kernel).
__global__ void __launch_bounds__(kPackWarps * 32)
    pack_vel_kernel(const double *__restrict__ vel, const int32_t *__restrict__ perm,
                    const ClusterDev *__restrict__ cls, const int32_t *__restrict__ tile_cluster,
                    int tc, int64_t n, int n_tiles, float *pvx, float *pvy, float *pvz,
                    float4 *vchl) {
    const int lane = threadIdx.x % 32;
    const int t = blockIdx.x * kPackWarps + threadIdx.x / 32;
    if (t >= n_tiles) return;
    const ClusterDev cl = cls[tile_cluster[t]];
    const int base = t * tc;
    const int per = tc / 32;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int r = 0; r < per; ++r) {
        const int slot = base + lane + 32 * r;
        if (slot - cl.slot_begin < cl.n) {
            const int64_t u = perm[slot];
            s[0] += vel[u];
            s[1] += vel[n + u];
            s[2] += vel[2 * n + u];
            s[3] += 1.0;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    const double cnt = s[3] > 0.0 ? s[3] : 1.0;
    const double cx = s[0] / cnt, cy = s[1] / cnt, cz = s[2] / cnt;
#pragma unroll 4
    for (int r = 0; r < per; ++r) {
        const int slot = base + lane + 32 * r;
        if (slot - cl.slot_begin < cl.n) {
            const int64_t u = perm[slot];
            pvx[slot] = (float)(vel[u] - cx);
            pvy[slot] = (float)(vel[n + u] - cy);
            pvz[slot] = (float)(vel[2 * n + u] - cz);
        } else {
            pvx[slot] = pvy[slot] = pvz[slot] = 0.0f;
        }
    }
    if (lane == 0) {
        const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
        vchl[2 * t + 0] = make_float4(hx, hy, hz, 0.0f);
        vchl[2 * t + 1] = make_float4((float)(cx - hx), (float)(cy - hy), (float)(cz - hz), 0.0f);
    }
}

__global__ void hermite_predict_kernel(int64_t n3, const double *__restrict__ pos,
                                       const double *__restrict__ vel,
                                       const double *__restrict__ acc,
                                       const double *__restrict__ jerk, double dt,
                                       double *__restrict__ xp, double *__restrict__ vp) {
    const double dt2 = dt * dt, dt3 = dt2 * dt;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x) {
        xp[q] = pos[q] + vel[q] * dt + acc[q] * dt2 / 2.0 + jerk[q] * dt3 / 6.0;
        vp[q] = vel[q] + acc[q] * dt + jerk[q] * dt2 / 2.0;
    }
}

__global__ void hermite_correct_kernel(int64_t n3, double *__restrict__ pos,
                                       double *__restrict__ vel, double *__restrict__ acc,
                                       double *__restrict__ jerk, const double *__restrict__ a1,
                                       const double *__restrict__ j1, double dt) {
    const double dt2 = dt * dt;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double a0 = acc[q], j0 = jerk[q], v0 = vel[q];
        const double v1 = v0 + (a0 + a1[q]) * dt / 2.0 + (j0 - j1[q]) * dt2 / 12.0;
        pos[q] = pos[q] + (v0 + v1) * dt / 2.0 + (a0 - a1[q]) * dt2 / 12.0;
        vel[q] = v1;
        acc[q] = a1[q];
        jerk[q] = j1[q];
    }
}

// v += half_dt * a; x += dt * v over the 3n entries of the SoA arrays.
__global__ void kick_drift_kernel(int64_t n3, double *__restrict__ pos, double *__restrict__ vel,
                                  const double *__restrict__ acc, double half_dt, double dt) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double v = vel[q] + half_dt * acc[q];
        vel[q] = v;
        pos[q] += dt * v;
    }
}

constexpr int kEnergyThreads = 256;

// Stage 1: per chunk, K, W, Px, Py, Pz, Lx, Ly, Lz (each a fixed-order sum).
__global__ void __launch_bounds__(kEnergyThreads)
    energy_chunk_kernel(const double *__restrict__ pos, const double *__restrict__ vel,
                        const double *__restrict__ mass, const double *__restrict__ pot, int64_t n,
                        const Chunk *__restrict__ chunks, double *__restrict__ part) {
    __shared__ double red[kEnergyThreads / 32][8];
    const Chunk ch = chunks[blockIdx.x];
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int64_t i = ch.begin + threadIdx.x; i < ch.end; i += kEnergyThreads) {
        const double m = mass[i];
        const double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
        const double vx = vel[i], vy = vel[n + i], vz = vel[2 * n + i];
        v[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        v[1] += pot ? 0.5 * m * pot[i] : 0.0;
        v[2] += m * vx;
        v[3] += m * vy;
        v[4] += m * vz;
        v[5] += m * (y * vz - z * vy);
        v[6] += m * (z * vx - x * vz);
        v[7] += m * (x * vy - y * vx);
    }
    block_sum<kEnergyThreads, 8>(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) part[8 * blockIdx.x + k] = v[k];
}

// Stage 2: one thread per cluster adds its chunks in order.
__global__ void energy_cluster_kernel(const double *__restrict__ part,
                                      const int32_t *__restrict__ chunk_first, int ncl,
                                      double *out_base, int *counter) {
    double *out = out_base;
    if (counter) out += (int64_t)(*counter) * ncl * 9;
    for (int c = threadIdx.x; c < ncl; c += blockDim.x) {
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = chunk_first[c]; k < chunk_first[c + 1]; ++k)
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] += part[8 * k + q];
        double *o = out + 9 * c;
        o[0] = v[0];
        o[1] = v[1];
        o[2] = v[0] + v[1];
#pragma unroll
        for (int q = 0; q < 6; ++q) o[3 + q] = v[2 + q];
    }
    __syncthreads();
    if (counter && threadIdx.x == 0) *counter += 1;
}

__global__ void check_finite_kernel(const double *__restrict__ a, int64_t n3,
                                    const double *__restrict__ b, int64_t n, int *flag) {
    bool bad = false;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3 + n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double v = q < n3 ? a[q] : (b ? b[q - n3] : 0.0);
        bad |= !isfinite(v);
    }
    if (bad) atomicExch(flag, 1);
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_pack(int n_tiles, const PackParams &prm, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    if (prm.tc % 32 != 0) return cudaErrorInvalidValue;
    pack_kernel<<<(n_tiles + kPackWarps - 1) / kPackWarps, kPackWarps * 32, 0, s>>>(prm, n_tiles);
    return cudaGetLastError();
}

cudaError_t launch_pack_vel(int n_tiles, const double *vel, const int32_t *perm,
                            const ClusterDev *cl, const int32_t *tile_cluster, int tc, int64_t n,
                            float *pvx, float *pvy, float *pvz, float4 *vchl, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    if (tc % 32 != 0) return cudaErrorInvalidValue;
    pack_vel_kernel<<<(n_tiles + kPackWarps - 1) / kPackWarps, kPackWarps * 32, 0, s>>>(
        vel, perm, cl, tile_cluster, tc, n, n_tiles, pvx, pvy, pvz, vchl);
    return cudaGetLastError();
}

cudaError_t launch_hermite_predict(int64_t n3, const double *pos, const double *vel,
                                   const double *acc, const double *jerk, double dt, double *xp,
                                   double *vp, cudaStream_t s) {
    if (n3 <= 0) return cudaSuccess;
    hermite_predict_kernel<<<grid_for(n3, 256), 256, 0, s>>>(n3, pos, vel, acc, jerk, dt, xp, vp);
    return cudaGetLastError();
}

cudaError_t launch_hermite_correct(int64_t n3, double *pos, double *vel, double *acc, double *jerk,
                                   const double *a1, const double *j1, double dt, cudaStream_t s) {
    if (n3 <= 0) return cudaSuccess;
    hermite_correct_kernel<<<grid_for(n3, 256), 256, 0, s>>>(n3, pos, vel, acc, jerk, a1, j1, dt);
    return cudaGetLastError();
}

cudaError_t launch_kick_drift(int64_t n3, double *pos, double *vel, const double *acc,
                              double half_dt, double dt, cudaStream_t s) {
    if (n3 <= 0) return cudaSuccess;
    kick_drift_kernel<<<grid_for(n3, 256), 256, 0, s>>>(n3, pos, vel, acc, half_dt, dt);
    return cudaGetLastError();
}

cudaError_t launch_energy(const double *pos, const double *vel, const double *mass,
                          const double *pot, int64_t n, const Chunk *chunks, int n_chunks,
                          const int32_t *chunk_first, int ncl, double *part, double *out_base,
                          int *counter, cudaStream_t s) {
    if (n_chunks > 0) {
        energy_chunk_kernel<<<n_chunks, kEnergyThreads, 0, s>>>(pos, vel, mass, pot, n, chunks,
                                                                 part);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    energy_cluster_kernel<<<1, 256, 0, s>>>(part, chunk_first, ncl, out_base, counter);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double *acc, int64_t n3, const double *pot, int64_t n,
                                int *flag, cudaStream_t s) {
    if (n3 + n <= 0) return cudaSuccess;
    check_finite_kernel<<<grid_for(n3 + n, 256), 256, 0, s>>>(acc, n3, pot, pot ? n : 0, flag);
    return cudaGetLastError();
}

}  // namespace nbody
