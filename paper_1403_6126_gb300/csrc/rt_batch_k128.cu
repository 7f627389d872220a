// Persistent multi-problem kernel, 128 threads per CTA: tiles of 128 (1-D),
// 16x8 (2-D) and 8x4x4 (3-D) cells.
#include "rt_batch_kernel.cuh"

namespace rtg {

BatchVariant batch_variant_128() { return BatchImpl<128, 16, 8, 8, 4, 4>::describe(); }

}  // namespace rtg
