// f32c_inst_c.cu -- instantiations of the F32C force kernel (split across
// translation units so they compile in parallel).
#include "f32c_shapes.h"
#include "forces_f32c.cuh"

namespace nbody {

#define SHAPE(B, P, T)                                                      \
    F32CShape{B, P, T, false, (const void *)forces_f32c_kernel<B, P, T, false>}, \
        F32CShape{B, P, T, true, (const void *)forces_f32c_kernel<B, P, T, true>}

extern const F32CShape kShapesC[] = {SHAPE(256, 4, 512), SHAPE(128, 8, 512), SHAPE(256, 1, 256), SHAPE(128, 4, 512)};
extern const int kNumShapesC = sizeof(kShapesC) / sizeof(kShapesC[0]);

}  // namespace nbody
