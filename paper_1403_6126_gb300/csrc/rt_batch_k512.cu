// Persistent multi-problem kernel, 512 threads per CTA: tiles of 512 (1-D),
// 32x16 (2-D) and 16x8x4 (3-D) cells.
#include "rt_batch_kernel.cuh"

namespace rtg {

BatchVariant batch_variant_512() { return BatchImpl<512, 32, 16, 16, 8, 4>::describe(); }

}  // namespace rtg
