// Tile shapes (cells per CTA along x, y, z; one thread per cell) compiled
// for each precision and grid dimension, preferred shape first.  A larger
// tile stages a smaller halo per cell but needs more shared memory (in the
// double-precision kernel a per-cell angle array grows with the angle
// count, so big angle sets fall back to smaller tiles); the smallest shapes
// (32 threads) spread small grids over more SMs.  rt_autotune times the
// shapes that fit.  X-macro lists: X(tx, ty, tz).
#pragma once

#include "rt_internal.h"

#define RT_SHAPES_F3(X) X(8, 8, 4) X(16, 8, 4) X(8, 4, 4) X(4, 4, 4)
#define RT_SHAPES_F2(X) X(32, 16, 1) X(16, 16, 1) X(16, 8, 1) X(8, 8, 1) X(8, 4, 1)
#define RT_SHAPES_F1(X) X(512, 1, 1) X(256, 1, 1) X(128, 1, 1) X(64, 1, 1) X(32, 1, 1)
#define RT_SHAPES_D3(X) X(8, 8, 4) X(8, 4, 4) X(4, 4, 4)
#define RT_SHAPES_D2(X) X(16, 16, 1) X(16, 8, 1) X(8, 8, 1) X(8, 4, 1)
#define RT_SHAPES_D1(X) X(256, 1, 1) X(128, 1, 1) X(64, 1, 1) X(32, 1, 1)

namespace rtg {
namespace stepk {
template <int P>
struct QTable;
}
// Launchers of the compiled shapes, one translation unit per group; they
// return cudaErrorInvalidConfiguration for a shape that is not compiled.
// qt: the launch-parameter table of the float kernel, or NULL for angle sets
// beyond it (the table is then built in shared memory).
cudaError_t launch_f3(const StepArgs<float> &a, const stepk::QTable<40> *qt, bool vel, TileShape t, cudaStream_t s);
cudaError_t launch_f12(const StepArgs<float> &a, const stepk::QTable<40> *qt, int dim, bool vel, TileShape t,
                       cudaStream_t s);
cudaError_t launch_d(const StepArgs<double> &a, int dim, bool vel, TileShape t, cudaStream_t s);
}  // namespace rtg
