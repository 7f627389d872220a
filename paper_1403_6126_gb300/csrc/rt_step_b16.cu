// Instantiations of the fused float step kernel with bf16 intensity storage
// (RT_BF16): the default tile of each dimension.
#include "rt_step_pair.cuh"

namespace rtg {

cudaError_t launch_b16(const StepArgs<float> &a, int dim, bool vel, TileShape t, cudaStream_t s) {
  if (dim == 3 && t.tx == 16 && t.ty == 8 && t.tz == 4)
    return vel ? stepk::launch_shape2<3, true, 16, 8, 4, true>(a, s) : stepk::launch_shape2<3, false, 16, 8, 4, true>(a, s);
  if (dim == 2 && t.tx == 32 && t.ty == 16 && t.tz == 1)
    return vel ? stepk::launch_shape2<2, true, 32, 16, 1, true>(a, s) : stepk::launch_shape2<2, false, 32, 16, 1, true>(a, s);
  if (dim == 1 && t.tx == 512 && t.ty == 1 && t.tz == 1)
    return vel ? stepk::launch_shape2<1, true, 512, 1, 1, true>(a, s) : stepk::launch_shape2<1, false, 512, 1, 1, true>(a, s);
  return cudaErrorInvalidConfiguration;
}

}  // namespace rtg
