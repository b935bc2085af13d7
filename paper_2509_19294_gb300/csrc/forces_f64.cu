// forces_f64.cu -- plain FP64 direct-summation kernel (the comparator path).
//
// Same quantity as the F32C kernel (Sec. 3 force sum divided by m_i, Plummer
// softened), every operation in IEEE double, straight from the caller's
// arrays: one i-particle per thread, j-particles staged through shared memory
// in tiles of kF64Block, one CTA per (cluster, block of i).  The self pair is
// masked by index; with eps = 0, coincident distinct particles contribute 0.
// GB300's FP64 rate is a small fraction of its FP32 rate, so this path exists
// for accuracy comparisons, not speed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nbody_internal.h"

namespace nbody {

namespace {

__global__ void __launch_bounds__(kF64Block) forces_f64_kernel(const F64Params p) {
    __shared__ double sj[4][kF64Block];
    const int2 blk = p.blocks[blockIdx.x];
    const ClusterDev cl = p.cl[blk.x];
    const int li = blk.y + threadIdx.x;
    const bool active = li < cl.n;
    const int64_t i = cl.user_begin + (active ? li : 0);
    const double xi = p.pos[i], yi = p.pos[p.n + i], zi = p.pos[2 * p.n + i];
    double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
    for (int j0 = 0; j0 < cl.n; j0 += kF64Block) {
        const int lj = j0 + threadIdx.x;
        __syncthreads();
        if (lj < cl.n) {
            const int64_t j = cl.user_begin + lj;
            sj[0][threadIdx.x] = p.pos[j];
            sj[1][threadIdx.x] = p.pos[p.n + j];
            sj[2][threadIdx.x] = p.pos[2 * p.n + j];
            sj[3][threadIdx.x] = p.mass[j];
        }
        __syncthreads();
        const int cnt = min(kF64Block, cl.n - j0);
        for (int k = 0; k < cnt; ++k) {
            const double dx = sj[0][k] - xi;
            const double dy = sj[1][k] - yi;
            const double dz = sj[2][k] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz + cl.eps2;
            const bool skip = (j0 + k == li) || !(r2 > 0.0);
            const double s = skip ? 0.0 : rsqrt(r2);
            const double ms = sj[3][k] * s;
            const double w3 = ms * s * s;
            ph += ms;
            ax += w3 * dx;
            ay += w3 * dy;
            az += w3 * dz;
        }
    }
    if (!active) return;
    const double a0 = p.G * ax, a1 = p.G * ay, a2 = p.G * az;
    p.acc[i] = a0;
    p.acc[p.n + i] = a1;
    p.acc[2 * p.n + i] = a2;
    if (p.pot) p.pot[i] = -p.G * ph;
    if (p.vel) {
        p.vel[i] += p.half_dt * a0;
        p.vel[p.n + i] += p.half_dt * a1;
        p.vel[2 * p.n + i] += p.half_dt * a2;
    }
}

// Acceleration, jerk and potential in FP64 (same structure; velocities from velin).
__global__ void __launch_bounds__(kF64Block) forces_jerk_f64_kernel(const F64Params p) {
    __shared__ double sj[7][kF64Block];
    const int2 blk = p.blocks[blockIdx.x];
    const ClusterDev cl = p.cl[blk.x];
    const int li = blk.y + threadIdx.x;
    const bool active = li < cl.n;
    const int64_t i = cl.user_begin + (active ? li : 0);
    const double xi = p.pos[i], yi = p.pos[p.n + i], zi = p.pos[2 * p.n + i];
    const double vxi = p.velin[i], vyi = p.velin[p.n + i], vzi = p.velin[2 * p.n + i];
    double ax = 0.0, ay = 0.0, az = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, ph = 0.0;
    for (int j0 = 0; j0 < cl.n; j0 += kF64Block) {
        const int lj = j0 + threadIdx.x;
        __syncthreads();
        if (lj < cl.n) {
            const int64_t j = cl.user_begin + lj;
            sj[0][threadIdx.x] = p.pos[j];
            sj[1][threadIdx.x] = p.pos[p.n + j];
            sj[2][threadIdx.x] = p.pos[2 * p.n + j];
            sj[3][threadIdx.x] = p.mass[j];
            sj[4][threadIdx.x] = p.velin[j];
            sj[5][threadIdx.x] = p.velin[p.n + j];
            sj[6][threadIdx.x] = p.velin[2 * p.n + j];
        }
        __syncthreads();
        const int cnt = min(kF64Block, cl.n - j0);
        for (int k = 0; k < cnt; ++k) {
            const double dx = sj[0][k] - xi, dy = sj[1][k] - yi, dz = sj[2][k] - zi;
            const double ux = sj[4][k] - vxi, uy = sj[5][k] - vyi, uz = sj[6][k] - vzi;
            const double r2 = dx * dx + dy * dy + dz * dz + cl.eps2;
            const bool skip = (j0 + k == li) || !(r2 > 0.0);
            const double s = skip ? 0.0 : rsqrt(r2);
            const double ms = sj[3][k] * s;
            const double s2 = s * s;
            const double w3 = ms * s2;
            const double beta = -3.0 * (dx * ux + dy * uy + dz * uz) * s2;
            ph += ms;
            ax += w3 * dx;
            ay += w3 * dy;
            az += w3 * dz;
            jx += w3 * (ux + beta * dx);
            jy += w3 * (uy + beta * dy);
            jz += w3 * (uz + beta * dz);
        }
    }
    if (!active) return;
    p.acc[i] = p.G * ax;
    p.acc[p.n + i] = p.G * ay;
    p.acc[2 * p.n + i] = p.G * az;
    p.jerk[i] = p.G * jx;
    p.jerk[p.n + i] = p.G * jy;
    p.jerk[2 * p.n + i] = p.G * jz;
    if (p.pot) p.pot[i] = -p.G * ph;
}

}  // namespace

cudaError_t launch_f64(int grid, const F64Params &prm, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    if (prm.jerk) {
        if (!prm.velin) return cudaErrorInvalidValue;
        forces_jerk_f64_kernel<<<grid, kF64Block, 0, s>>>(prm);
    } else {
        forces_f64_kernel<<<grid, kF64Block, 0, s>>>(prm);
    }
    return cudaGetLastError();
}

}  // namespace nbody
