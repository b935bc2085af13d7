// block_reduce.cuh -- deterministic CTA-wide sums.
#pragma once

#include <cuda_runtime.h>

namespace nbody {

// Sum of NV doubles over a CTA of NT threads in a fixed order (shuffle tree in
// each warp, then the warps in order), so the result is bitwise reproducible;
// every thread receives the totals.  scratch: __shared__ double[NT / 32][NV].
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

}  // namespace nbody
