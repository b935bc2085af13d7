// kernels_misc.cu -- pack, leapfrog, diagnostics and finiteness kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "block_reduce.cuh"
#include "nbody_internal.h"

namespace nbody {

namespace {

// One CTA per centre tile: FP32 offsets of the tile's particles from its
// centre, FP32 masses; pad slots get mass 0 and a far offset.  The centre is
// the mean of the FP32-rounded positions, summed in FP32 in a fixed order (so
// bitwise reproducible); any point near the tile serves, since the offsets are
// FP64 differences from it rounded once, and FP64 work is scarce on this part
// (one FP32 reduction instead of an FP64 one and six divisions per thread).
// The centre is stored as a float pair (hi, lo = 0) for the force kernels.
// With VEL the velocities are packed the same way (pads get offset 0).
template <int NT, bool VEL>
__global__ void __launch_bounds__(NT) pack_kernel(const PackParams p) {
    constexpr int NV = VEL ? 7 : 4;
    __shared__ float red[NT / 32][NV];
    __shared__ float cen[6];
    const int t = blockIdx.x;
    const ClusterDev cl = p.cl[p.tile_cluster[t]];
    const int base = t * p.tc;
    const int per = p.tc / NT;
    float s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = 0.0f;
    for (int r = 0; r < per; ++r) {
        const int slot = base + threadIdx.x + NT * r;
        if (slot - cl.slot_begin < cl.n) {
            const int64_t u = p.perm[slot];
#pragma unroll
            for (int d = 0; d < 3; ++d) s[d] += (float)p.pos[d * p.n + u];
            s[3] += 1.0f;
            if (VEL)
#pragma unroll
                for (int d = 0; d < 3; ++d) s[4 + d] += (float)p.vel[d * p.n + u];
        }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if (threadIdx.x % 32 == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[threadIdx.x / 32][k] = s[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            float v = red[0][k];
            for (int w = 1; w < NT / 32; ++w) v += red[w][k];
            s[k] = v;
        }
        const float inv = s[3] > 0.0f ? 1.0f / s[3] : 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cen[d] = s[d] * inv;
            cen[3 + d] = VEL ? s[4 + d] * inv : 0.0f;
        }
        p.chl[2 * t + 0] = make_float4(cen[0], cen[1], cen[2], 0.0f);
        p.chl[2 * t + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (VEL) {
            p.vchl[2 * t + 0] = make_float4(cen[3], cen[4], cen[5], 0.0f);
            p.vchl[2 * t + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    __syncthreads();
    double c[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) c[d] = (double)cen[d];
    for (int r = 0; r < per; ++r) {
        const int slot = base + threadIdx.x + NT * r;
        if (slot - cl.slot_begin < cl.n) {
            const int64_t u = p.perm[slot];
            p.px[slot] = (float)(p.pos[u] - c[0]);
            p.py[slot] = (float)(p.pos[p.n + u] - c[1]);
            p.pz[slot] = (float)(p.pos[2 * p.n + u] - c[2]);
            p.pm[slot] = (float)p.mass[u];
            if (VEL) {
                p.pvx[slot] = (float)(p.vel[u] - c[3]);
                p.pvy[slot] = (float)(p.vel[p.n + u] - c[4]);
                p.pvz[slot] = (float)(p.vel[2 * p.n + u] - c[5]);
            }
        } else {
            p.px[slot] = kPadOffset;
            p.py[slot] = kPadOffset;
            p.pz[slot] = kPadOffset;
            p.pm[slot] = 0.0f;
            if (VEL) p.pvx[slot] = p.pvy[slot] = p.pvz[slot] = 0.0f;
        }
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
    if (prm.tc <= 0 || prm.tc % 128 != 0) return cudaErrorInvalidValue;
    const bool vel = prm.vel != nullptr;
    if (prm.tc % 256 == 0) {
        if (vel) pack_kernel<256, true><<<n_tiles, 256, 0, s>>>(prm);
        else pack_kernel<256, false><<<n_tiles, 256, 0, s>>>(prm);
    } else {
        if (vel) pack_kernel<128, true><<<n_tiles, 128, 0, s>>>(prm);
        else pack_kernel<128, false><<<n_tiles, 128, 0, s>>>(prm);
    }
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
