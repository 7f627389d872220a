// Instantiations of the two-kernel 3-D step (rt_split.cuh), float
// intensities, one per x-y column tile of the transport kernel.
#include "rt_shapes.h"
#include "rt_split.cuh"

namespace rtg {

cudaError_t launch_split(const StepArgs<float> &a, bool vel, TileShape t, cudaStream_t s) {
  if (t.tz != 0 || !a.scr_w || !a.scr_face) return cudaErrorInvalidValue;
#define RT_CASE(X, Y)                                                            \
  if (t.tx == X && t.ty == Y) return vel ? split::launch<true, X, Y>(a, s) : split::launch<false, X, Y>(a, s);
  RT_SHAPES_S3(RT_CASE)
#undef RT_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace rtg
