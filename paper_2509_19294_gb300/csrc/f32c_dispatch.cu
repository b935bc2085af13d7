// f32c_dispatch.cu -- lookup, occupancy and launch of the compiled F32C shapes.
#include <cuda_runtime.h>

#include "f32c_shapes.h"
#include "nbody_internal.h"

namespace nbody {

namespace {

constexpr int kTables = 4;
const F32CShape *const kTab[kTables] = {kShapesA, kShapesB, kShapesC, kShapesD};
const int *const kCnt[kTables] = {&kNumShapesA, &kNumShapesB, &kNumShapesC, &kNumShapesD};

// minb == 0 matches the first compiled variant of (block, p, tj).
const F32CShape *find_shape(int block, int p, int tj, int minb, bool eps_zero) {
    for (int t = 0; t < kTables; ++t)
        for (int k = 0; k < *kCnt[t]; ++k) {
            const F32CShape &s = kTab[t][k];
            if (s.block == block && s.p == p && s.tj == tj && s.eps_zero == eps_zero &&
                (minb == 0 || s.minb == minb))
                return &s;
        }
    return nullptr;
}

}  // namespace

int f32c_shapes(int *block, int *p, int *tj, int *minb, int cap) {
    int n = 0;
    for (int t = 0; t < kTables; ++t)
        for (int k = 0; k < *kCnt[t]; ++k) {
            const F32CShape &s = kTab[t][k];
            if (s.eps_zero) continue;
            if (n < cap) {
                block[n] = s.block;
                p[n] = s.p;
                tj[n] = s.tj;
                minb[n] = s.minb;
            }
            ++n;
        }
    return n;
}

int f32c_resolve_minb(int block, int p, int tj, int minb, bool eps_zero) {
    const F32CShape *s = find_shape(block, p, tj, minb, eps_zero);
    return s ? s->minb : 0;
}

int f32c_occupancy(int block, int p, int tj, int minb, bool eps_zero) {
    const F32CShape *s = find_shape(block, p, tj, minb, eps_zero);
    if (!s) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, s->kernel, block, 0) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_f32c(int block, int p, int tj, int minb, bool eps_zero, int grid,
                        const F32CParams &prm, cudaStream_t st) {
    const F32CShape *s = find_shape(block, p, tj, minb, eps_zero);
    if (!s) return cudaErrorNotSupported;
    if (grid <= 0) return cudaSuccess;
    void *args[] = {(void *)&prm};
    return cudaLaunchKernel(s->kernel, dim3(grid), dim3(block), args, 0, st);
}

}  // namespace nbody
