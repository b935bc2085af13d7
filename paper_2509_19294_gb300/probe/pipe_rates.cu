// pipe_rates.cu -- per-SM issue-rate probes behind the force kernel's roofline
// (libnbody_probe.so, a measurement library for the benchmark; not part of the
// force library's ABI).
//
// The roofline of the F32C force kernel is set by the FP32 pipe (13 FP32
// operations per pair) and the MUFU rsqrt unit (1 per pair).  These probes run
// one CTA of 1024 threads per SM and count cycles with clock64(), so each rate
// is per SM per clock and independent of the clock frequency:
//   * FP32: independent chains of paired FMA (__ffma2_rn), lane-operations.
//   * MUFU: independent chains of rsqrt.approx.ftz.f32.
//   * pair: the force kernel's own per-pair arithmetic (F32CKernel::body, its
//           potential terms added as a tree of four as in the tile loop) on
//           register-resident data whose j operands change every call
//           (4 extra paired ops per 8 pairs), i.e. a lower bound on its
//           ceiling without shared loads; one CTA of 256 threads per SM, as
//           the kernel's C5 shapes run.
//   * FP64: independent chains of fma(double).
#include <cuda_runtime.h>
#include <stdint.h>

#include "forces_f32c.cuh"
#include "pipe_rates.h"

namespace nbody {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) ffma2_probe(int iters, float *sink,
                                                             long long *cycles) {
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(threadIdx.x * 1e-3f + k, k * 0.5f);
    const float2 b = make_float2(0.999f, 1.001f), c = make_float2(1e-6f, -1e-6f);
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b, c);
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kProbeThreads) rsqrt_probe(int iters, float *sink,
                                                             long long *cycles) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + threadIdx.x * 1e-4f + k;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = rsqrt_mufu(a[k]);
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kProbeThreads) dfma_probe(int iters, float *sink,
                                                            long long *cycles) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3 + k;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], 0.999, 1e-6);
    __syncthreads();
    const long long t1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// The force kernel's pair arithmetic with P = 4 i-particles per thread and
// j-particles taken from registers (varied every iteration so nothing folds).
constexpr int kPairP = 4;
using PairK = F32CKernel<256, kPairP, 512, false>;

// One CTA of 256 threads per SM with up to 255 registers, as the kernel's C5
// shape (256, 4, 512 or 1024) runs.
constexpr int kPairThreads = 256;
__global__ void __launch_bounds__(kPairThreads, 1) pair_probe(int iters, float *sink,
                                                              long long *cycles) {
    float2 nx[kPairP], ny[kPairP], nz[kPairP], ax[kPairP], ay[kPairP], az[kPairP], ph[kPairP];
#pragma unroll
    for (int k = 0; k < kPairP; ++k) {
        const float q = threadIdx.x * 1e-3f + k * 0.37f;
        nx[k] = make_float2(-q, -q);
        ny[k] = make_float2(0.5f * q, 0.5f * q);
        nz[k] = make_float2(-0.25f * q, -0.25f * q);
        ax[k] = ay[k] = az[k] = ph[k] = make_float2(0.0f, 0.0f);
    }
    const float2 e2 = make_float2(1e-6f, 1e-6f);
    // four independent j-pairs per iteration (the kernel loads them from
    // shared memory, so they do not depend on each other)
    float2 xj[4], yj[4], zj[4], mj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        xj[q] = make_float2(0.1f + 0.01f * q, 0.2f);
        yj[q] = make_float2(-0.3f, 0.4f + 0.01f * q);
        zj[q] = make_float2(0.5f, -0.6f - 0.01f * q);
        mj[q] = make_float2(1e-3f, 2e-3f);
    }
    const float2 dj = make_float2(1e-4f, -1e-4f);
    const int dself[kPairP] = {-1, -1, -1, -1};  // no self pair among the probe's j's
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        // the potential terms of the four j-pairs added as a tree, as the
        // kernel's tile loop does
        float2 m[4][kPairP];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            PairK::body<false>(xj[q], yj[q], zj[q], mj[q], e2, nx, ny, nz, ax, ay, az, m[q], dself, 0);
#pragma unroll
        for (int k = 0; k < kPairP; ++k)
            ph[k] = __fadd2_rn(ph[k], __fadd2_rn(__fadd2_rn(m[0][k], m[1][k]), __fadd2_rn(m[2][k], m[3][k])));
        // every j operand changes each iteration, so nothing can be hoisted;
        // these 4 paired ops per 2 * kPairP pairs make the figure a lower bound
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            xj[q] = __fadd2_rn(xj[q], dj);
            yj[q] = __fadd2_rn(yj[q], dj);
            zj[q] = __fadd2_rn(zj[q], dj);
            mj[q] = __fmul2_rn(mj[q], make_float2(1.0001f, 0.9999f));
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPairP; ++k) s += ax[k].x + ay[k].y + az[k].x + ph[k].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace nbody

extern "C" int nbody_measure_pipes(double *out, int n_out) {
    using namespace nbody;
    if (!out || n_out < 4) return NBODY_PROBE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return NBODY_PROBE_ECUDA;
    }
    float *sink = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * sms * kProbeThreads) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(long long) * sms) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sink);
        return NBODY_PROBE_ENOMEM;
    }
    const int iters = 4096;
    long long *hc = new long long[sms];
    double rate[4];
    int rc = 0;
    for (int probe = 0; probe < 4 && rc == 0; ++probe) {
        for (int rep = 0; rep < 2; ++rep) {  // first launch warms up
            switch (probe) {
                case 0: ffma2_probe<<<sms, kProbeThreads>>>(iters, sink, cyc); break;
                case 1: rsqrt_probe<<<sms, kProbeThreads>>>(iters, sink, cyc); break;
                case 2: pair_probe<<<sms, kPairThreads>>>(iters / 4, sink, cyc); break;
                default: dfma_probe<<<sms, kProbeThreads>>>(iters / 16, sink, cyc); break;
            }
        }
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(hc, cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            rc = NBODY_PROBE_ECUDA;
            break;
        }
        double mean = 0.0;
        for (int k = 0; k < sms; ++k) mean += (double)hc[k];
        mean /= sms;
        const double threads = kProbeThreads;
        switch (probe) {
            case 0: rate[0] = threads * iters * kChains * 2.0 / mean; break;
            case 1: rate[1] = threads * iters * kChains / mean; break;
            case 2: rate[2] = kPairThreads * (double)(iters / 4) * (4 * 2.0 * kPairP) / mean; break;
            default: rate[3] = threads * (iters / 16) * kChains / mean; break;
        }
    }
    delete[] hc;
    cudaFree(sink);
    cudaFree(cyc);
    if (rc == 0)
        for (int k = 0; k < 4; ++k) out[k] = rate[k];
    return rc;
}
