// Persistent multi-problem step kernel (see rt_batch.cu): CTAs walk the
// (problem, tile) work list in a fixed interleave and run the same per-tile
// code as the single-problem float kernel.  One compiled variant per
// tile set; all shapes of a set have the same thread count (one per cell).
#pragma once

#include "rt_step_quad.cuh"

namespace rtg {

struct WorkItem {
  int prob, tbx, tby, tbz;
};

// Host-side description of a compiled variant.
struct BatchVariant {
  int threads;
  TileShape t1, t2, t3;   // tiles of 1-D, 2-D and 3-D members
  cudaError_t (*prepare)(bool vel, size_t smem, int *blocks_per_sm);
  cudaError_t (*launch)(bool vel, int grid, size_t smem, const StepArgs<float> *descs, const WorkItem *items,
                        int nitems, cudaStream_t s);
};

constexpr int kBatchVariants = 3;
// Variants in order: 512, 256 and 128 threads per CTA.
const BatchVariant &batch_variant(int i);

template <bool VEL, int NT, int X2, int Y2, int X3, int Y3, int Z3>
__global__ void __launch_bounds__(NT, 512 / NT)
    batch_kernel(const StepArgs<float> *__restrict__ descs, const WorkItem *__restrict__ items, int nitems) {
  static_assert(X2 * Y2 == NT && X3 * Y3 * Z3 == NT, "every tile shape has one thread per cell");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ StepArgs<float> desc;
  const int tid = threadIdx.x;
  // CTA b takes items b, b + grid, b + 2 grid, ...: the list is sorted by
  // decreasing cost, so every CTA gets a like share, and no claim (atomic,
  // barrier, broadcast) stands between one tile and the next
  int cur = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    if (w.prob != cur) {   // the descriptor is copied only when the problem changes
      __syncthreads();     // every thread is done with the previous one
      const int *src = reinterpret_cast<const int *>(descs + w.prob);
      int *dst = reinterpret_cast<int *>(&desc);
      for (int i = tid; i < (int)(sizeof(StepArgs<float>) / sizeof(int)); i += NT) dst[i] = src[i];
      __syncthreads();
      cur = w.prob;
    }
    if (desc.dim == 3)
      stepk::process_tile_q<3, VEL, X3, Y3, Z3, false, 2>(desc, nullptr, tid, w.tbx, w.tby, w.tbz, smem);
    else if (desc.dim == 2)
      stepk::process_tile_q<2, VEL, X2, Y2, 1, false, 2>(desc, nullptr, tid, w.tbx, w.tby, 0, smem);
    else
      stepk::process_tile_q<1, VEL, NT, 1, 1, false, 2>(desc, nullptr, tid, w.tbx, 0, 0, smem);
  }
}

template <int NT, int X2, int Y2, int X3, int Y3, int Z3>
struct BatchImpl {
  static cudaError_t prepare(bool vel, size_t smem, int *per_sm) {
    auto kern = vel ? batch_kernel<true, NT, X2, Y2, X3, Y3, Z3> : batch_kernel<false, NT, X2, Y2, X3, Y3, Z3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, NT, smem);
  }
  static cudaError_t launch(bool vel, int grid, size_t smem, const StepArgs<float> *descs, const WorkItem *items,
                            int nitems, cudaStream_t s) {
    auto kern = vel ? batch_kernel<true, NT, X2, Y2, X3, Y3, Z3> : batch_kernel<false, NT, X2, Y2, X3, Y3, Z3>;
    kern<<<grid, NT, smem, s>>>(descs, items, nitems);
    return cudaGetLastError();
  }
  static BatchVariant describe() {
    return BatchVariant{NT, TileShape{NT, 1, 1}, TileShape{X2, Y2, 1}, TileShape{X3, Y3, Z3}, &prepare, &launch};
  }
};

BatchVariant batch_variant_512();
BatchVariant batch_variant_256();
BatchVariant batch_variant_128();

}  // namespace rtg
