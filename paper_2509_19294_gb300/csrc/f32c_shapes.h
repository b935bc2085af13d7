// f32c_shapes.h -- table of compiled F32C force-kernel instantiations.
#pragma once

namespace nbody {

struct F32CShape {
    int block, p, tj, minb;
    bool eps_zero;
    const void *kernel;  // __global__ void(F32CParams)
};

extern const F32CShape kShapesA[];
extern const int kNumShapesA;
extern const F32CShape kShapesB[];
extern const int kNumShapesB;
extern const F32CShape kShapesC[];
extern const int kNumShapesC;
extern const F32CShape kShapesD[];
extern const int kNumShapesD;

}  // namespace nbody
