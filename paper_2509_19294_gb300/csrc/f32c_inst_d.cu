// f32c_inst_d.cu -- instantiations of the F32C force kernel (split across
// translation units so they compile in parallel).  SHAPE(block, p, tj, ctas_per_sm).
#include "f32c_shapes.h"
#include "forces_f32c.cuh"

namespace nbody {

#define SHAPE(B, P, T, M)                                                              \
    F32CShape{B, P, T, M, false, (const void *)forces_f32c_kernel<B, P, T, M, false>}, \
        F32CShape{B, P, T, M, true, (const void *)forces_f32c_kernel<B, P, T, M, true>}

extern const F32CShape kShapesD[] = {SHAPE(64, 2, 128, 8), SHAPE(64, 4, 256, 6)};
extern const int kNumShapesD = sizeof(kShapesD) / sizeof(kShapesD[0]);

}  // namespace nbody
