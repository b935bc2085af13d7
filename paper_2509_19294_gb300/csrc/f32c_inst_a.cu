// f32c_inst_a.cu -- instantiations of the F32C force kernel (split across
// translation units so they compile in parallel).
#include "f32c_shapes.h"
#include "forces_f32c.cuh"

namespace nbody {

#define SHAPE(B, P, T)                                                      \
    F32CShape{B, P, T, false, (const void *)forces_f32c_kernel<B, P, T, false>}, \
        F32CShape{B, P, T, true, (const void *)forces_f32c_kernel<B, P, T, true>}

extern const F32CShape kShapesA[] = {SHAPE(128, 4, 256), SHAPE(256, 2, 256), SHAPE(128, 2, 256)};
extern const int kNumShapesA = sizeof(kShapesA) / sizeof(kShapesA[0]);

}  // namespace nbody
