// Internal layout of a context (one problem), shared by the single-problem
// runtime (rt_api.cu), the multi-problem runtime (rt_batch.cu) and the
// serving loop (rt_server.cpp).
#pragma once

#include <string>
#include <vector>

#include "rt.h"
#include "rt_internal.h"

struct rt_ctx {
  int dim = 0, n[3] = {1, 1, 1}, M = 0;
  long long N = 0;
  double dx[3] = {1, 1, 1};
  int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  double C = 1, P = 1;
  rt_options opt{};
  cudaStream_t stream = nullptr;
  bool fp64 = false;
  bool bf16 = false;  // intensities stored as bf16 deviations (RT_BF16)
  size_t rs = 4;      // bytes per stored real of the cell data (rho, sigma, v)
  size_t rsI = 4;     // bytes per stored intensity
  bool quad = false;  // float intensities in the quad-interleaved layout (RT_FP32)
  size_t I_bytes = 0; // bytes of one intensity buffer
  float *qscr = nullptr;  // bf16 storage: float [M][N] scratch for Q_m
  float *cen[2] = {nullptr, nullptr};   // float step: each cell's smallest intensity over angles [N]
  bool has_v = false, material_set = false, intensity_set = false;
  rtg::TileShape tile{0, 0, 0};
  // device state (Real = double or float)
  void *I[2] = {nullptr, nullptr};
  double *mom[2] = {nullptr, nullptr};   // E, F, P [10][N], double for every precision
  int cur = 0;
  void *rho = nullptr, *sa = nullptr, *ss = nullptr, *v = nullptr;
  double *T = nullptr, *dEgas = nullptr;
  double *dMom = nullptr;                 // Delta(rho v) [3][N]
  void *ang = nullptr, *inflow = nullptr;
  int *flags = nullptr;  // [0] Newton failures, [1] input scan
  double *stage = nullptr;
  long long stage_len = 0;
  std::vector<double> host_n, host_w, host_inflow;
  // the angle table [M][4] and inflow table [6][M] rounded to float, as the
  // device tables hold them (launch-parameter tables of the float kernel)
  std::vector<float> host_angf, host_inflowf;
  // captured multi-step graph
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0;
  int graph_steps = 0, graph_cur = -1;
  bool graph_vel = false;
  void *batch = nullptr;  // the rt_batch this context belongs to, if any
  // rt_step_coupled: copy streams (fields in, sources out), a stream for the
  // field conversions, a second stream for every other slab's kernel, and
  // the events that order them against the slab launches, made on first use
  static constexpr int kSlabs = 8;
  cudaStream_t xs_in = nullptr, xs_out = nullptr, xs_cv = nullptr, xs_k = nullptr;
  cudaEvent_t ev_start = nullptr, ev_copied[kSlabs] = {}, ev_in[kSlabs] = {}, ev_done[kSlabs] = {};
};

#include <nvtx3/nvToolsExt.h>

namespace rtg {
// Device allocation of the library: cudaMalloc, unless rt_fault_inject has
// armed a failure for this allocation.
cudaError_t device_alloc(void **p, size_t bytes);
// NVTX range over an entry point (free when no profiler is attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};
// Step arguments of context c for its current buffer parity.
template <typename Real>
StepArgs<Real> make_args(rt_ctx *c, double dt);
// Whether the velocity terms are on (v != 0 somewhere, or the estimate).
bool velocity_on(const rt_ctx *c);
// Records msg as this thread's last error and returns s.
rt_status set_error(rt_status s, const std::string &msg);
// RT_OK, or RT_E_INVALID (message prefixed by `where`) when the Newton
// options of o are out of range.
rt_status check_newton_options(const rt_options &o, const char *where);
// Device bytes rt_create allocates for N cells and M angles.
size_t context_bytes(long long N, int M, bool fp64);
// Launch of the fused step for context c (its host tables feed the float
// kernel's launch-parameter table).
cudaError_t launch_ctx_step(rt_ctx *c, const StepArgs<float> &a, bool vel, TileShape t);
cudaError_t launch_ctx_step(rt_ctx *c, const StepArgs<double> &a, bool vel, TileShape t);
// The same on stream s instead of the context's stream.
cudaError_t launch_ctx_step_on(rt_ctx *c, const StepArgs<float> &a, bool vel, TileShape t, cudaStream_t s);
cudaError_t launch_ctx_step_on(rt_ctx *c, const StepArgs<double> &a, bool vel, TileShape t, cudaStream_t s);
// Whether a problem of this dimension and angle count fits the batch tile.
bool batch_fits(int dim, int M, bool vel);
// Marks a batch for a rebuild before its next step (a member changed what
// the batch's launch depends on).
void batch_touch(void *batch);
}  // namespace rtg
