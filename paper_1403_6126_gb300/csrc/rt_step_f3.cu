// Instantiations of the fused step kernel (two angles per thread): float, 3-D shapes.
#include "rt_shapes.h"
#include "rt_step_pair.cuh"

namespace rtg {

cudaError_t launch_f3(const StepArgs<float> &a, bool vel, TileShape t, cudaStream_t s) {
#define RT_CASE(X, Y, Z)                                                          \
  if (t.tx == X && t.ty == Y && t.tz == Z)                                        \
    return vel ? stepk::launch_shape2<3, true, X, Y, Z>(a, s)               \
               : stepk::launch_shape2<3, false, X, Y, Z>(a, s);
  RT_SHAPES_F3(RT_CASE)
#undef RT_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace rtg
