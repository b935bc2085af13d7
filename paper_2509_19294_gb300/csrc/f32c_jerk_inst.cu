// f32c_jerk_inst.cu -- instantiations, lookup, occupancy and launch of the
// acceleration + jerk kernel.  SHAPE(block, p, tj, ctas_per_sm).
#include <cuda_runtime.h>

#include "forces_f32c_jerk.cuh"
#include "nbody_internal.h"

namespace nbody {

namespace {

struct JerkShape {
    int block, p, tj, minb;
    bool eps_zero;
    const void *kernel;
};

#define SHAPE(B, P, T, M)                                                                   \
    JerkShape{B, P, T, M, false, (const void *)forces_f32c_jerk_kernel<B, P, T, M, false>}, \
        JerkShape{B, P, T, M, true, (const void *)forces_f32c_jerk_kernel<B, P, T, M, true>}

const JerkShape kJerkShapes[] = {SHAPE(128, 2, 256, 2), SHAPE(256, 2, 256, 1), SHAPE(256, 2, 512, 1),
                                 SHAPE(128, 1, 128, 4), SHAPE(64, 2, 128, 4), SHAPE(128, 2, 128, 3)};

const JerkShape *find(int block, int p, int tj, int minb, bool eps_zero) {
    for (const JerkShape &s : kJerkShapes)
        if (s.block == block && s.p == p && s.tj == tj && s.eps_zero == eps_zero &&
            (minb == 0 || s.minb == minb))
            return &s;
    return nullptr;
}

}  // namespace

int f32c_jerk_shapes(int *block, int *p, int *tj, int *minb, int cap) {
    int n = 0;
    for (const JerkShape &s : kJerkShapes) {
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

int f32c_jerk_resolve_minb(int block, int p, int tj, int minb, bool eps_zero) {
    const JerkShape *s = find(block, p, tj, minb, eps_zero);
    return s ? s->minb : 0;
}

int f32c_jerk_occupancy(int block, int p, int tj, int minb, bool eps_zero) {
    const JerkShape *s = find(block, p, tj, minb, eps_zero);
    if (!s) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, s->kernel, block, 0) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_f32c_jerk(int block, int p, int tj, int minb, bool eps_zero, int grid,
                             const F32CJerkParams &prm, cudaStream_t st) {
    const JerkShape *s = find(block, p, tj, minb, eps_zero);
    if (!s) return cudaErrorNotSupported;
    if (grid <= 0) return cudaSuccess;
    void *args[] = {(void *)&prm};
    return cudaLaunchKernel(s->kernel, dim3(grid), dim3(block), args, 0, st);
}

}  // namespace nbody
