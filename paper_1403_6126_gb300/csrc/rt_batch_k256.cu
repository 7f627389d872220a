// Persistent multi-problem kernel, 256 threads per CTA: tiles of 256 (1-D),
// 16x16 (2-D) and 8x8x4 (3-D) cells.
#include "rt_batch_kernel.cuh"

namespace rtg {

BatchVariant batch_variant_256() { return BatchImpl<256, 16, 16, 8, 8, 4>::describe(); }

}  // namespace rtg
