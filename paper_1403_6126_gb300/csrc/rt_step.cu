// Tile choice and dispatch of the fused step kernels (rt_step_quad.cuh for
// float intensities, rt_step_pair.cuh for their bf16 storage,
// rt_step_kernel.cuh for double): the compiled shapes are listed in
// rt_shapes.h.
#include "rt_shapes.h"
#include "rt_step_quad.cuh"

namespace rtg {

namespace {

template <typename Real>
int shape_list(int dim, TileShape *out) {
  int n = 0;
#define RT_ADD(X, Y, Z) out[n++] = TileShape{X, Y, Z};
  if (sizeof(Real) == 4) {
    if (dim == 1) { RT_SHAPES_F1(RT_ADD) }
    else if (dim == 2) { RT_SHAPES_F2(RT_ADD) }
    else { RT_SHAPES_F3(RT_ADD) }
  } else {
    if (dim == 1) { RT_SHAPES_D1(RT_ADD) }
    else if (dim == 2) { RT_SHAPES_D2(RT_ADD) }
    else { RT_SHAPES_D3(RT_ADD) }
  }
#undef RT_ADD
  return n;
}

// Shared memory of a shape within the opt-in limit: the quad kernel for
// float (its pair table in the launch parameters up to 80 angles), the
// scalar kernel for double.
template <typename Real>
bool fits(int dim, int M, bool has_v, TileShape t) {
  const size_t sm = sizeof(Real) == 4
                        ? stepk::smem_bytes_q(dim, M, has_v, t.tx, t.ty, t.tz, M <= 2 * stepk::kQTabPairsSmall)
                        : stepk::smem_bytes(dim, M, has_v, t.tx, t.ty, t.tz, sizeof(Real));
  return sm <= 227 * 1024;
}

}  // namespace

template <typename Real>
int tile_candidates(int dim, int M, bool has_v, TileShape *out) {
  TileShape list[16];
  int n = shape_list<Real>(dim, list), k = 0;
  for (int i = 0; i < n; ++i)
    if (fits<Real>(dim, M, has_v, list[i])) out[k++] = list[i];
  return k;
}

template <typename Real>
bool tile_ok(int dim, int M, bool has_v, TileShape t) {
  TileShape list[16];
  int n = shape_list<Real>(dim, list);
  for (int i = 0; i < n; ++i)
    if (list[i].tx == t.tx && list[i].ty == t.ty && list[i].tz == t.tz)
      return fits<Real>(dim, M, has_v, t);
  return false;
}

template <typename Real>
bool choose_tile(int dim, int M, bool has_v, TileShape *out) {
  TileShape list[16];
  int n = shape_list<Real>(dim, list);
  for (int i = 0; i < n; ++i) {
    if (fits<Real>(dim, M, has_v, list[i])) {
      *out = list[i];
      return true;
    }
  }
  return false;
}

bool choose_tile_b16(int dim, int M, TileShape *out) {
  const TileShape t = dim == 3 ? TileShape{16, 8, 4} : dim == 2 ? TileShape{32, 16, 1} : TileShape{512, 1, 1};
  if (stepk::smem_bytes2(dim, M, true, t.tx, t.ty, t.tz) > 227 * 1024) return false;
  *out = t;
  return true;
}

template <>
cudaError_t launch_step<float>(const StepArgs<float> &a, int dim, bool has_v, TileShape t, cudaStream_t s) {
  return launch_b16(a, dim, has_v, t, s);
}

cudaError_t launch_step_quad(const StepArgs<float> &a, const float *host_ang, const float *host_inflow, int dim,
                             bool vel, TileShape t, cudaStream_t s) {
  if (a.M <= 2 * stepk::kQTabPairsSmall) {
    stepk::QTable<stepk::kQTabPairsSmall> qt;
    stepk::fill_qtable(&qt, host_ang, a.M, a.C, a.dtdx, host_inflow);
    return dim == 3 ? launch_f3(a, &qt, vel, t, s) : launch_f12(a, &qt, dim, vel, t, s);
  }
  return dim == 3 ? launch_f3(a, nullptr, vel, t, s) : launch_f12(a, nullptr, dim, vel, t, s);
}

template <>
cudaError_t launch_step<double>(const StepArgs<double> &a, int dim, bool has_v, TileShape t, cudaStream_t s) {
  return launch_d(a, dim, has_v, t, s);
}

template bool choose_tile<float>(int, int, bool, TileShape *);
template bool choose_tile<double>(int, int, bool, TileShape *);
template bool tile_ok<float>(int, int, bool, TileShape);
template int tile_candidates<float>(int, int, bool, TileShape *);
template int tile_candidates<double>(int, int, bool, TileShape *);
template bool tile_ok<double>(int, int, bool, TileShape);

}  // namespace rtg
