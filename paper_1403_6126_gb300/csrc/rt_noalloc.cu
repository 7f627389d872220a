// One radiation step without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or under a strict memory budget, plugins that may
// only touch buffers handed to them, and latency-critical paths where an
// allocation could block or fail.  rt_step_noalloc serves them: the caller
// passes every field as a device pointer, the angle and inflow tables travel
// in the kernel's launch parameters, and the one word of scratch the
// persistent step kernel needs (the count of cells whose T^4 Newton failed)
// lives in a fixed file-scope device array, reserved once per GPU when the
// library is loaded and kept until the process exits.  The launch-parameter
// table bounds the angle count to kNoallocMaxAngles.
//
// The array is shared by every call: each call clears the failure word before
// its kernel runs, so nothing carries over from the previous call, but two
// calls that overlap on the GPU (different streams without ordering between
// them) race on it.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "rt.h"
#include "rt_ctx.h"
#include "rt_step_quad.cuh"

namespace rtg {

namespace {

constexpr int kNoallocMaxAngles = 2 * stepk::kQTabPairsLarge;   // 256
// the failure word and a reserved word, padded to the array's alignment
constexpr size_t kNoallocScratchBytes = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

using NoallocTable = stepk::QTable<stepk::kQTabPairsLarge>;

// Persistent tiles of one problem: CTA b takes tiles b, b + grid, b + 2 grid,
// ... (the tiles cost alike, so no claim has to stand between one tile and
// the next).
template <int DIM, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ, stepk::kQMinBlocks<TX * TY * TZ>)
    noalloc_kernel(const StepArgs<float> a, const __grid_constant__ NoallocTable qt) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ntx = (a.n[0] + TX - 1) / TX, nty = (a.n[1] + TY - 1) / TY, ntz = (a.n[2] + TZ - 1) / TZ;
  const int ntiles = ntx * nty * ntz;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x)
    stepk::process_tile_q<DIM, true, TX, TY, TZ, true, stepk::kQTabPairsLarge>(
        a, &qt, threadIdx.x, it % ntx, (it / ntx) % nty, it / (ntx * nty), smem);
}

// Per device: the scratch array's device address, and per dimension the SM
// count and resident CTAs at the shared-memory size last set.
struct DeviceCache {
  void *scratch = nullptr;
  int sms = 0;
  size_t smem[3] = {0, 0, 0};
  int per_sm[3] = {0, 0, 0};
};
struct NoallocState {
  std::mutex mu;
  DeviceCache dev[64];
};
NoallocState g_state;

rt_status current_device(int *dev) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return set_error(RT_E_CUDA, std::string("rt_step_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  if (*dev < 0 || *dev >= 64) return set_error(RT_E_INVALID, "rt_step_noalloc: device ordinal above 63");
  return RT_OK;
}

// The scratch address for the current device (looked up on its first call,
// with the device current).
rt_status scratch_for(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lock(g_state.mu);
  DeviceCache &d = g_state.dev[dev];
  if (!d.scratch) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(RT_E_CUDA, std::string("rt_step_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
      return set_error(RT_E_CUDA, std::string("rt_step_noalloc: SM count: ") + cudaGetErrorString(e));
    d.scratch = p;
    d.sms = std::max(1, sms);
  }
  *out = static_cast<unsigned char *>(d.scratch);
  return RT_OK;
}

template <int DIM, int TX, int TY, int TZ>
cudaError_t launch_noalloc(const StepArgs<float> &a, const NoallocTable &qt, int dev, cudaStream_t s) {
  const size_t sm = stepk::smem_bytes_q(DIM, a.M, true, TX, TY, TZ, true);
  auto kern = noalloc_kernel<DIM, TX, TY, TZ>;
  int per_sm = 0, sms = 0;
  {
    // the attribute and the occupancy are set / asked only when the shared
    // memory grows past what this device's kernel of this dimension has seen
    std::lock_guard<std::mutex> lock(g_state.mu);
    DeviceCache &d = g_state.dev[dev];
    if (sm > d.smem[DIM - 1]) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.per_sm[DIM - 1], kern, TX * TY * TZ, sm);
      if (e != cudaSuccess) return e;
      d.smem[DIM - 1] = sm;
    }
    per_sm = std::max(1, d.per_sm[DIM - 1]);
    sms = d.sms;
  }
  const long long ntiles = (long long)((a.n[0] + TX - 1) / TX) * ((a.n[1] + TY - 1) / TY) * ((a.n[2] + TZ - 1) / TZ);
  const int grid = (int)std::max(1LL, std::min(ntiles, (long long)sms * per_sm));
  kern<<<grid, TX * TY * TZ, sm, s>>>(a, qt);
  return cudaGetLastError();
}

}  // namespace

}  // namespace rtg

extern "C" rt_status rt_step_noalloc(const rt_grid *g, const rt_angles *ang, double Crat, double Prat,
                                     const rt_options *opts, double dt, const rt_noalloc_fields *f,
                                     int *newton_failures) {
  using rtg::set_error;
  if (!g || !ang || !ang->n || !ang->w || !opts || !f) return set_error(RT_E_INVALID, "rt_step_noalloc: NULL argument");
  if (!f->I_in || !f->I_out || !f->rho || !f->sigma_a || !f->sigma_s || !f->v || !f->T || !f->mom_in ||
      !f->mom_out || !f->dE_gas || !f->dMom)
    return set_error(RT_E_INVALID, "rt_step_noalloc: NULL field pointer");
  if ((const void *)f->I_in == (const void *)f->I_out || (const void *)f->mom_in == (const void *)f->mom_out)
    return set_error(RT_E_INVALID, "rt_step_noalloc: I_in / I_out and mom_in / mom_out must be different buffers");
  if (g->dim < 1 || g->dim > 3) return set_error(RT_E_INVALID, "rt_step_noalloc: dim must be 1, 2 or 3");
  const int M = ang->m;
  if (M < 1 || M > rtg::kNoallocMaxAngles)
    return set_error(RT_E_INVALID, "rt_step_noalloc: angle count outside 1..256 (the launch-parameter table holds 256)");
  long long N = 1;
  rtg::StepArgs<float> a;
  a.dim = g->dim;
  for (int d = 0; d < 3; ++d) {
    const bool act = d < g->dim;
    a.n[d] = act ? g->n[d] : 1;
    if (act && (g->n[d] < 1 || !(g->hi[d] > g->lo[d])))
      return set_error(RT_E_INVALID, "rt_step_noalloc: empty grid axis");
    if (act && (g->bc[d][0] < RT_BC_PERIODIC || g->bc[d][0] > RT_BC_INFLOW || g->bc[d][1] < RT_BC_PERIODIC ||
                g->bc[d][1] > RT_BC_INFLOW || (g->bc[d][0] == RT_BC_PERIODIC) != (g->bc[d][1] == RT_BC_PERIODIC)))
      return set_error(RT_E_INVALID, "rt_step_noalloc: bad boundary kinds");
    a.bc[d][0] = act ? g->bc[d][0] : RT_BC_PERIODIC;
    a.bc[d][1] = act ? g->bc[d][1] : RT_BC_PERIODIC;
    const double dx = act ? (g->hi[d] - g->lo[d]) / g->n[d] : 1.0;
    a.dx[d] = (float)dx;
    a.dtdx[d] = (float)(dt / dx);
    N *= a.n[d];
  }
  if (N >= (1LL << 28)) return set_error(RT_E_INVALID, "rt_step_noalloc: more than 2^28 cells");
  if (!(dt > 0) || !std::isfinite(dt) || !(Crat > 0) || !(Prat > 0) || !(opts->gamma > 1) || !(opts->r_ideal > 0) ||
      !std::isfinite(Crat) || !std::isfinite(Prat) || !std::isfinite(opts->gamma) || !std::isfinite(opts->r_ideal))
    return set_error(RT_E_INVALID, "rt_step_noalloc: need finite dt, Crat, Prat, r_ideal > 0 and gamma > 1");
  if (opts->precision != RT_FP32) return set_error(RT_E_INVALID, "rt_step_noalloc: float intensities only (RT_FP32)");
  if (rt_status st = rtg::check_newton_options(*opts, "rt_step_noalloc"); st != RT_OK) return st;
  const size_t sm_need = g->dim == 1   ? rtg::stepk::smem_bytes_q(1, M, true, 512, 1, 1, true)
                         : g->dim == 2 ? rtg::stepk::smem_bytes_q(2, M, true, 32, 16, 1, true)
                                       : rtg::stepk::smem_bytes_q(3, M, true, 8, 8, 4, true);
  if (sm_need > 227 * 1024) return set_error(RT_E_INVALID, "rt_step_noalloc: too many angles for one tile's shared memory");
  double wsum = 0;
  for (int m = 0; m < M; ++m) {
    const double *nm = ang->n + 3 * m;
    if (!(std::fabs(std::sqrt(nm[0] * nm[0] + nm[1] * nm[1] + nm[2] * nm[2]) - 1.0) <= 1e-12) || !(ang->w[m] > 0))
      return set_error(RT_E_INVALID, "rt_step_noalloc: angles need |n| = 1 and W > 0");
    wsum += ang->w[m];
  }
  if (!(std::fabs(wsum - 1.0) <= 1e-12)) return set_error(RT_E_INVALID, "rt_step_noalloc: weights must sum to 1");
  cudaStream_t s = (cudaStream_t)opts->stream;
  if (newton_failures) {
    // the count is read back with a blocking copy, which a stream under
    // capture cannot take
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return set_error(RT_E_CUDA, std::string("rt_step_noalloc: ") + cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
      return set_error(RT_E_INVALID, "rt_step_noalloc: newton_failures must be NULL on a stream that is capturing");
  }

  int dev = 0;
  rt_status st = rtg::current_device(&dev);
  if (st != RT_OK) return st;
  unsigned char *scratch = nullptr;
  if ((st = rtg::scratch_for(dev, &scratch)) != RT_OK) return st;
  int *counter = reinterpret_cast<int *>(scratch);

  // the angle table as the device would round it, and the inflow table
  float angf[4 * rtg::kNoallocMaxAngles], inflowf[6 * rtg::kNoallocMaxAngles];
  for (int m = 0; m < M; ++m) {
    for (int d = 0; d < 3; ++d) angf[4 * m + d] = (float)ang->n[3 * m + d];
    angf[4 * m + 3] = (float)ang->w[m];
  }
  for (int i = 0; i < 6 * M; ++i) inflowf[i] = f->inflow ? (float)f->inflow[i] : 0.0f;
  a.M = M;
  a.N = N;
  a.C = (float)Crat;
  a.invC = (float)(1.0 / Crat);
  a.P = (float)Prat;
  a.dt = (float)dt;
  a.dt_d = dt;
  a.kv_per_rho = opts->r_ideal / (opts->gamma - 1.0);
  a.hold_T = opts->hold_T;
  a.estimate_v = opts->estimate_v;
  a.newton_max_it = opts->newton_max_it;
  a.newton_rtol = opts->newton_rtol;
  a.wnorm = rtg::weight_norm(angf, M);
  rtg::table_moment_sums(angf, M, a.msum);
  a.ang = nullptr;      // the launch-parameter table replaces both
  a.inflow = nullptr;
  a.I_in = f->I_in;
  a.I_out = f->I_out;
  a.rho = f->rho;
  a.sa = f->sigma_a;
  a.ss = f->sigma_s;
  a.v = f->v;
  a.T_in = f->T;
  a.T_out = f->T;
  a.mom_in = f->mom_in;
  a.mom_out = f->mom_out;
  a.cen_in = nullptr;   // cell centers formed from I_in in the kernel
  a.cen_out = nullptr;
  a.dEgas = f->dE_gas;
  a.dMom = f->dMom;
  a.status = counter;
  a.I16_in = nullptr;
  a.I16_out = nullptr;
  a.Q = nullptr;
  a.outer_begin = 0;
  a.outer_count = 0;
  rtg::NoallocTable qt;   // 22 KB, passed by value as the launch parameters
  rtg::stepk::fill_qtable(&qt, angf, M, a.C, a.dtdx, inflowf);

  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);   // the failure word
  if (e != cudaSuccess) return set_error(RT_E_CUDA, std::string("rt_step_noalloc: clear: ") + cudaGetErrorString(e));
  e = g->dim == 1   ? rtg::launch_noalloc<1, 512, 1, 1>(a, qt, dev, s)
      : g->dim == 2 ? rtg::launch_noalloc<2, 32, 16, 1>(a, qt, dev, s)
                    : rtg::launch_noalloc<3, 8, 8, 4>(a, qt, dev, s);
  if (e != cudaSuccess) return set_error(RT_E_CUDA, std::string("rt_step_noalloc: launch: ") + cudaGetErrorString(e));
  if (newton_failures) {
    e = cudaMemcpyAsync(newton_failures, counter, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(RT_E_CUDA, std::string("rt_step_noalloc: status read: ") + cudaGetErrorString(e));
  }
  return RT_OK;
}
