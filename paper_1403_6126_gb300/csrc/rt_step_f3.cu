// Instantiations of the fused float step kernel (quad layout, two angles per
// thread per phase): 3-D shapes.
#include "rt_shapes.h"
#include "rt_step_quad.cuh"

namespace rtg {

cudaError_t launch_f3(const StepArgs<float> &a, const stepk::QTable<40> *qt, bool vel, TileShape t, cudaStream_t s) {
#define RT_CASE(X, Y, Z)                                                          \
  if (t.tx == X && t.ty == Y && t.tz == Z)                                        \
    return vel ? stepk::launch_shape_q<3, true, X, Y, Z>(a, qt, s)                \
               : stepk::launch_shape_q<3, false, X, Y, Z>(a, qt, s);
  RT_SHAPES_F3(RT_CASE)
#undef RT_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace rtg
