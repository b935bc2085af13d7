// f32c_inst_b.cu -- instantiations of the F32C force kernel (split across
// translation units so they compile in parallel).
#include "f32c_shapes.h"
#include "forces_f32c.cuh"

namespace nbody {

#define SHAPE(B, P, T)                                                      \
    F32CShape{B, P, T, false, (const void *)forces_f32c_kernel<B, P, T, false>}, \
        F32CShape{B, P, T, true, (const void *)forces_f32c_kernel<B, P, T, true>}

extern const F32CShape kShapesB[] = {SHAPE(64, 4, 256), SHAPE(128, 1, 128), SHAPE(64, 2, 128)};
extern const int kNumShapesB = sizeof(kShapesB) / sizeof(kShapesB[0]);

}  // namespace nbody
