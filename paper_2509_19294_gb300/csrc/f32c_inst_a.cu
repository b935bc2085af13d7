// f32c_inst_a.cu -- instantiations of the F32C force kernel (split across
// translation units so they compile in parallel).  SHAPE(block, p, tj, ctas_per_sm).
#include "f32c_shapes.h"
#include "forces_f32c.cuh"

namespace nbody {

#define SHAPE(B, P, T, M)                                                              \
    F32CShape{B, P, T, M, false, (const void *)forces_f32c_kernel<B, P, T, M, false>}, \
        F32CShape{B, P, T, M, true, (const void *)forces_f32c_kernel<B, P, T, M, true>}

extern const F32CShape kShapesA[] = {SHAPE(256, 2, 256, 2), SHAPE(128, 2, 256, 4), SHAPE(256, 4, 1024, 1)};
extern const int kNumShapesA = sizeof(kShapesA) / sizeof(kShapesA[0]);

}  // namespace nbody
