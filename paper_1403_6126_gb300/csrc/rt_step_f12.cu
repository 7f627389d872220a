// Instantiations of the fused float step kernel (quad layout, two angles per
// thread per phase): 1-D and 2-D shapes.
#include "rt_shapes.h"
#include "rt_step_quad.cuh"

namespace rtg {

cudaError_t launch_f12(const StepArgs<float> &a, const stepk::QTable<40> *qt, int dim, bool vel, TileShape t,
                       cudaStream_t s) {
#define RT_CASE(D, X, Y, Z)                                                       \
  if (dim == D && t.tx == X && t.ty == Y && t.tz == Z)                            \
    return vel ? stepk::launch_shape_q<D, true, X, Y, Z>(a, qt, s)                \
               : stepk::launch_shape_q<D, false, X, Y, Z>(a, qt, s);
#define RT_CASE1(X, Y, Z) RT_CASE(1, X, Y, Z)
#define RT_CASE2(X, Y, Z) RT_CASE(2, X, Y, Z)
  RT_SHAPES_F1(RT_CASE1)
  RT_SHAPES_F2(RT_CASE2)
#undef RT_CASE1
#undef RT_CASE2
#undef RT_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace rtg
