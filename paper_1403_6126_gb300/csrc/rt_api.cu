// C ABI runtime: contexts, device state, validation, launches and graphs.
// The declarations and their documentation are in include/rt.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rt.h"
#include "rt_ctx.h"
#include "rt_internal.h"

namespace {

thread_local std::string g_last_error;

rt_status fail(rt_status s, const std::string &msg) {
  g_last_error = msg;
  return s;
}

}  // namespace

rt_status rtg::set_error(rt_status s, const std::string &msg) { return fail(s, msg); }

rt_status rtg::check_newton_options(const rt_options &o, const char *where) {
  if (o.newton_max_it < 1 || o.newton_max_it > 1000)
    return fail(RT_E_INVALID, std::string(where) + ": newton_max_it must be in 1..1000");
  if (!(o.newton_rtol >= 1e-15 && o.newton_rtol <= 1e-3))
    return fail(RT_E_INVALID, std::string(where) + ": newton_rtol must be in [1e-15, 1e-3]");
  return RT_OK;
}

namespace {
std::atomic<int> g_fail_alloc_after{-1};   // armed by rt_fault_inject
}

cudaError_t rtg::device_alloc(void **p, size_t bytes) {
  int k = g_fail_alloc_after.load();
  while (k >= 0) {
    if (g_fail_alloc_after.compare_exchange_weak(k, k - 1)) {
      if (k == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

namespace {

rt_status cuda_fail(cudaError_t e, const char *what) {
  return fail(RT_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RT_CUDA(call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

}  // namespace


namespace {

void free_all(rt_ctx *c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (cudaStream_t s : {c->xs_in, c->xs_cv, c->xs_out, c->xs_k}) {
    if (!s) continue;
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (c->ev_start) cudaEventDestroy(c->ev_start);
  for (int k = 0; k < rt_ctx::kSlabs; ++k) {
    if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
    if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
    if (c->ev_done[k]) cudaEventDestroy(c->ev_done[k]);
  }
  void *ptrs[] = {c->I[0], c->I[1], c->mom[0], c->mom[1], c->rho, c->sa, c->ss, c->v,
                  c->T, c->dEgas, c->dMom, c->ang, c->inflow, c->flags, c->stage, c->qscr, c->cen[0], c->cen[1]};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

}  // namespace

template <typename Real>
rtg::StepArgs<Real> rtg::make_args(rt_ctx *c, double dt) {
  rtg::StepArgs<Real> a;
  a.dim = c->dim;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = c->n[d];
    a.bc[d][0] = c->bc[d][0];
    a.bc[d][1] = c->bc[d][1];
    a.dx[d] = (Real)c->dx[d];
    a.dtdx[d] = (Real)(dt / c->dx[d]);
  }
  a.M = c->M;
  a.N = c->N;
  a.C = (Real)c->C;
  a.invC = (Real)(1.0 / c->C);
  a.P = (Real)c->P;
  a.dt = (Real)dt;
  a.dt_d = dt;
  a.kv_per_rho = c->opt.r_ideal / (c->opt.gamma - 1.0);
  a.hold_T = c->opt.hold_T;
  a.estimate_v = c->opt.estimate_v;
  a.newton_max_it = c->opt.newton_max_it;
  a.newton_rtol = c->opt.newton_rtol;
  a.wnorm = (Real)rtg::weight_norm(c->host_angf.data(), c->M);
  rtg::table_moment_sums(c->host_angf.data(), c->M, a.msum);
  a.ang = (const Real *)c->ang;
  a.inflow = (const Real *)c->inflow;
  a.I_in = (const Real *)c->I[c->cur];
  a.I_out = (Real *)c->I[1 - c->cur];
  a.I16_in = nullptr;
  a.I16_out = nullptr;
  a.Q = nullptr;
  if (c->bf16) {
    a.I_in = nullptr;
    a.I_out = nullptr;
    a.I16_in = (const unsigned short *)c->I[c->cur];
    a.I16_out = (unsigned short *)c->I[1 - c->cur];
    a.Q = c->qscr;
  }
  a.rho = (const Real *)c->rho;
  a.sa = (const Real *)c->sa;
  a.ss = (const Real *)c->ss;
  a.v = (const Real *)c->v;
  a.T_in = c->T;
  a.T_out = c->T;
  a.mom_in = c->mom[c->cur];
  a.mom_out = c->mom[1 - c->cur];
  a.cen_in = c->cen[c->cur];
  a.cen_out = c->cen[1 - c->cur];
  a.dEgas = c->dEgas;
  a.dMom = c->dMom;
  a.status = c->flags;
  a.outer_begin = 0;
  a.outer_count = 0;
  return a;
}

size_t rtg::context_bytes(long long N, int M, bool fp64) {
  const size_t rs = fp64 ? 8 : 4, Nz = (size_t)N, Mz = (size_t)M;
  const size_t Ms = fp64 ? Mz : 4 * (size_t)((M + 3) / 4);   // stored angles (float: quad padding)
  const size_t stage = sizeof(double) * std::max<size_t>(10 * Nz, 8 * Mz);
  const size_t centers = fp64 ? 0 : 2 * sizeof(float) * Nz;   // the float step's cell centers
  return rs * (2 * Ms * Nz + 6 * Nz + 10 * Mz) + 8 * (2 * 10 * Nz + 3 * Nz) + 16 * Nz + 2 * sizeof(int) + stage + centers;
}

cudaError_t rtg::launch_ctx_step_on(rt_ctx *c, const StepArgs<double> &a, bool vel, TileShape t, cudaStream_t s) {
  return launch_step<double>(a, c->dim, vel, t, s);
}

cudaError_t rtg::launch_ctx_step_on(rt_ctx *c, const StepArgs<float> &a, bool vel, TileShape t, cudaStream_t s) {
  if (c->bf16) return launch_step<float>(a, c->dim, vel, t, s);
  return launch_step_quad(a, c->host_angf.data(), c->host_inflowf.data(), c->dim, vel, t, s);
}

cudaError_t rtg::launch_ctx_step(rt_ctx *c, const StepArgs<double> &a, bool vel, TileShape t) {
  return launch_ctx_step_on(c, a, vel, t, c->stream);
}

cudaError_t rtg::launch_ctx_step(rt_ctx *c, const StepArgs<float> &a, bool vel, TileShape t) {
  return launch_ctx_step_on(c, a, vel, t, c->stream);
}

template rtg::StepArgs<float> rtg::make_args<float>(rt_ctx *, double);
template rtg::StepArgs<double> rtg::make_args<double>(rt_ctx *, double);

bool rtg::velocity_on(const rt_ctx *c) { return c->has_v || c->opt.estimate_v; }

namespace {

rt_status launch_step(rt_ctx *c, double dt) {
  cudaError_t e;
  bool vel = rtg::velocity_on(c);
  if (c->fp64)
    e = rtg::launch_ctx_step(c, rtg::make_args<double>(c, dt), vel, c->tile);
  else
    e = rtg::launch_ctx_step(c, rtg::make_args<float>(c, dt), vel, c->tile);
  if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
  c->cur = 1 - c->cur;
  return RT_OK;
}

rt_status convert_in(rt_ctx *c, const double *src, void *dst, long long n) {
  cudaError_t e = c->fp64 ? rtg::launch_convert_in<double>(src, (double *)dst, n, c->stream)
                          : rtg::launch_convert_in<float>(src, (float *)dst, n, c->stream);
  return e == cudaSuccess ? RT_OK : cuda_fail(e, "convert");
}

// Scan (and with convert, conversion into the context's arrays) of the gas
// fields staged in c->stage, cells [c0, c1); flag bits go to c->flags[1].
rt_status fields_in(rt_ctx *c, long long c0, long long c1, bool convert, cudaStream_t s) {
  cudaError_t e = c->fp64 ? rtg::launch_fields_in<double>(c->stage, c->N, c0, c1 - c0, convert, (double *)c->rho,
                                                          (double *)c->sa, (double *)c->ss, (double *)c->v, c->T,
                                                          c->flags + 1, s)
                          : rtg::launch_fields_in<float>(c->stage, c->N, c0, c1 - c0, convert, (float *)c->rho,
                                                         (float *)c->sa, (float *)c->ss, (float *)c->v, c->T,
                                                         c->flags + 1, s);
  return e == cudaSuccess ? RT_OK : cuda_fail(e, "fields");
}

rt_status convert_out(rt_ctx *c, const void *src, double *dst, long long n) {
  cudaError_t e = c->fp64 ? rtg::launch_convert_out<double>((const double *)src, dst, n, c->stream)
                          : rtg::launch_convert_out<float>((const float *)src, dst, n, c->stream);
  return e == cudaSuccess ? RT_OK : cuda_fail(e, "convert");
}

// Moments of the intensity just set (for bf16 storage: of the float field in
// the Q scratch, before encoding).
rt_status recompute_moments(rt_ctx *c) {
  const void *I = c->bf16 ? (const void *)c->qscr : c->I[c->cur];
  // the quad-layout float step takes its sums over the weights normalised
  // to sum 1, and so do these moments
  const double wscale = c->quad ? 1.0 / rtg::weight_sum(c->host_angf.data(), c->M) : 1.0;
  cudaError_t e = c->fp64 ? rtg::launch_moments<double>((const double *)I, (const double *)c->ang, c->M,
                                                        c->N, false, 1.0, c->mom[c->cur], c->stream)
                          : rtg::launch_moments<float>((const float *)I, (const float *)c->ang, c->M,
                                                       c->N, c->quad, wscale, c->mom[c->cur], c->stream);
  if (e == cudaSuccess && c->quad) e = rtg::launch_centers((const float *)I, c->M, c->N, c->cen[c->cur], c->stream);
  return e == cudaSuccess ? RT_OK : cuda_fail(e, "moments");
}

// Copies n doubles from the caller (host or device) into dst (device).
rt_status fetch(rt_ctx *c, const double *src, double *dst, long long n) {
  if (c->opt.device_ptrs) {
    RT_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    RT_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  return RT_OK;
}

// Queues the copy of n doubles from the device buffer src to the caller;
// delivered() then waits once for all of a call's copies to host memory.
rt_status deliver_async(rt_ctx *c, const double *src, double *dst, long long n) {
  RT_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double),
                          c->opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return RT_OK;
}

rt_status delivered(rt_ctx *c) {
  if (!c->opt.device_ptrs) RT_CUDA(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

// Copies n doubles from the device buffer src to the caller (host: waits).
rt_status deliver(rt_ctx *c, const double *src, double *dst, long long n) {
  rt_status st = deliver_async(c, src, dst, n);
  return st != RT_OK ? st : delivered(c);
}

}  // namespace

namespace {

// Copy streams and events of rt_step_coupled, made on first use (kept in the
// context as they are made, so free_all releases a partial set too).
rt_status coupled_init(rt_ctx *c) {
  if (c->xs_in && c->xs_out && c->xs_cv && c->xs_k && c->ev_done[rt_ctx::kSlabs - 1]) return RT_OK;
  if (!c->xs_k) RT_CUDA(cudaStreamCreateWithFlags(&c->xs_k, cudaStreamNonBlocking));
  if (!c->xs_in) RT_CUDA(cudaStreamCreateWithFlags(&c->xs_in, cudaStreamNonBlocking));
  if (!c->xs_out) RT_CUDA(cudaStreamCreateWithFlags(&c->xs_out, cudaStreamNonBlocking));
  if (!c->xs_cv) {
    // the field conversions run at the highest priority: the step's CTAs
    // fill every SM, and a conversion that waited for a whole slab to drain
    // would hold up the next slab
    int lo = 0, hi = 0;
    RT_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    RT_CUDA(cudaStreamCreateWithPriority(&c->xs_cv, cudaStreamNonBlocking, hi));
  }
  if (!c->ev_start) RT_CUDA(cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming));
  for (int k = 0; k < rt_ctx::kSlabs; ++k) {
    if (!c->ev_copied[k]) RT_CUDA(cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming));
    if (!c->ev_in[k]) RT_CUDA(cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming));
    if (!c->ev_done[k]) RT_CUDA(cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming));
  }
  return RT_OK;
}

// Fields of the cells [c0, c1) to the staging buffer (copy stream), in the
// layout rt_set_material uses: rho, T, v (3 components), sigma_a, sigma_s.
rt_status coupled_in(rt_ctx *c, const double *const f[5], long long c0, long long c1) {
  const long long N = c->N, n = c1 - c0;
  const size_t b = n * sizeof(double);
  const double *src[7] = {f[0], f[1], f[2], f[2] + N, f[2] + 2 * N, f[3], f[4]};
  for (int k = 0; k < 7; ++k)
    RT_CUDA(cudaMemcpyAsync(c->stage + k * N + c0, src[k] + c0, b, cudaMemcpyHostToDevice, c->xs_in));
  return RT_OK;
}

// Sources of the cells [c0, c1) back to the caller (all three double on the
// device), copied on the outgoing stream once ev (recorded after the slab's
// kernel on stream ks) has fired.
rt_status coupled_out(rt_ctx *c, long long c0, long long c1, cudaEvent_t ev, cudaStream_t ks, double *dE_gas,
                      double *dMom, double *T_new) {
  const long long N = c->N, n = c1 - c0;
  const double *s_mom = c->dMom;
  RT_CUDA(cudaEventRecord(ev, ks));
  RT_CUDA(cudaStreamWaitEvent(c->xs_out, ev, 0));
  const size_t b = n * sizeof(double);
  if (dE_gas) RT_CUDA(cudaMemcpyAsync(dE_gas + c0, c->dEgas + c0, b, cudaMemcpyDeviceToHost, c->xs_out));
  if (dMom)
    for (int i = 0; i < 3; ++i)
      RT_CUDA(cudaMemcpyAsync(dMom + i * N + c0, s_mom + i * N + c0, b, cudaMemcpyDeviceToHost, c->xs_out));
  if (T_new) RT_CUDA(cudaMemcpyAsync(T_new + c0, c->T + c0, b, cudaMemcpyDeviceToHost, c->xs_out));
  return RT_OK;
}

// The step's kernel over tile layers [l0, l1) along z (all layers: l1 = 0),
// on stream s.
rt_status coupled_launch(rt_ctx *c, double dt, bool vel, int l0, int l1, cudaStream_t s) {
  cudaError_t e;
  if (c->fp64) {
    rtg::StepArgs<double> a = rtg::make_args<double>(c, dt);
    a.outer_begin = l0;
    a.outer_count = l1 - l0;
    e = rtg::launch_ctx_step_on(c, a, vel, c->tile, s);
  } else {
    rtg::StepArgs<float> a = rtg::make_args<float>(c, dt);
    a.outer_begin = l0;
    a.outer_count = l1 - l0;
    e = rtg::launch_ctx_step_on(c, a, vel, c->tile, s);
  }
  return e == cudaSuccess ? RT_OK : cuda_fail(e, "step kernel launch");
}

}  // namespace

extern "C" {

const char *rt_last_error(void) { return g_last_error.c_str(); }

rt_status rt_fault_inject(int kind, int after) {
  if (kind == RT_FAULT_NONE) {
    g_fail_alloc_after.store(-1);
    return RT_OK;
  }
  if (kind != RT_FAULT_ALLOC || after < 0) return fail(RT_E_INVALID, "rt_fault_inject: unknown kind or after < 0");
  g_fail_alloc_after.store(after);
  return RT_OK;
}

rt_status rt_options_default(rt_options *o) {
  if (!o) return fail(RT_E_INVALID, "rt_options_default: NULL");
  std::memset(o, 0, sizeof(*o));
  o->precision = RT_FP32;
  o->cfl = 0.4;
  o->gamma = 5.0 / 3.0;
  o->r_ideal = 1.0;
  o->hold_T = 0;
  o->estimate_v = 1;
  o->device_ptrs = 0;
  o->stream = nullptr;
  o->newton_max_it = 60;
  o->newton_rtol = 1e-13;
  return RT_OK;
}

rt_status rt_create(const rt_grid *g, const rt_angles *ang, double Crat, double Prat, const rt_options *opts,
                    rt_ctx **out) {
  rtg::Range nvtx_range("rt_create");
  if (!out) return fail(RT_E_INVALID, "rt_create: out is NULL");
  *out = nullptr;
  if (!g || !ang || !ang->n || !ang->w) return fail(RT_E_INVALID, "rt_create: NULL grid or angles");
  if (g->dim < 1 || g->dim > 3) return fail(RT_E_INVALID, "rt_create: dim must be 1, 2 or 3");
  long long N = 1;
  for (int d = 0; d < 3; ++d) {
    int nd = d < g->dim ? g->n[d] : 1;
    if (d < g->dim) {
      if (nd < 1) return fail(RT_E_INVALID, "rt_create: n[d] < 1 on an active axis");
      if (!(g->hi[d] > g->lo[d]) || !std::isfinite(g->hi[d] - g->lo[d]))
        return fail(RT_E_INVALID, "rt_create: hi <= lo on an active axis");
      for (int s = 0; s < 2; ++s)
        if (g->bc[d][s] < RT_BC_PERIODIC || g->bc[d][s] > RT_BC_INFLOW)
          return fail(RT_E_INVALID, "rt_create: unknown boundary kind");
      if ((g->bc[d][0] == RT_BC_PERIODIC) != (g->bc[d][1] == RT_BC_PERIODIC))
        return fail(RT_E_INVALID, "rt_create: periodic must be set on both faces of an axis");
    }
    N *= nd;
  }
  if (N >= (1LL << 28)) return fail(RT_E_INVALID, "rt_create: more than 2^28 cells");
  int M = ang->m;
  if (M < 1 || M > rtg::kMaxAngles) return fail(RT_E_INVALID, "rt_create: angle count out of range (1..256)");
  double wsum = 0;
  for (int m = 0; m < M; ++m) {
    const double *nm = ang->n + 3 * m;
    double nn = nm[0] * nm[0] + nm[1] * nm[1] + nm[2] * nm[2];
    if (!(std::fabs(std::sqrt(nn) - 1.0) <= 1e-12)) return fail(RT_E_INVALID, "rt_create: |n| != 1");
    if (!(ang->w[m] > 0) || !std::isfinite(ang->w[m])) return fail(RT_E_INVALID, "rt_create: weight <= 0");
    wsum += ang->w[m];
  }
  if (!(std::fabs(wsum - 1.0) <= 1e-12)) return fail(RT_E_INVALID, "rt_create: weights must sum to 1");
  if (!(Crat > 0) || !(Prat > 0) || !std::isfinite(Crat) || !std::isfinite(Prat))
    return fail(RT_E_INVALID, "rt_create: Crat and Prat must be positive");
  rt_options o;
  rt_options_default(&o);
  if (opts) o = *opts;
  if (o.precision != RT_FP64 && o.precision != RT_FP32 && o.precision != RT_BF16)
    return fail(RT_E_INVALID, "rt_create: precision must be RT_FP64, RT_FP32 or RT_BF16");
  if (!(o.cfl > 0) || !(o.gamma > 1.0) || !(o.r_ideal > 0) || !std::isfinite(o.cfl) || !std::isfinite(o.gamma) ||
      !std::isfinite(o.r_ideal))
    return fail(RT_E_INVALID, "rt_create: need finite cfl > 0, gamma > 1, r_ideal > 0");
  if (rt_status st = rtg::check_newton_options(o, "rt_create"); st != RT_OK) return st;

  rt_ctx *c = new (std::nothrow) rt_ctx;
  if (!c) return fail(RT_E_NOMEM, "rt_create: host allocation");
  c->dim = g->dim;
  for (int d = 0; d < 3; ++d) {
    c->n[d] = d < g->dim ? g->n[d] : 1;
    c->dx[d] = d < g->dim ? (g->hi[d] - g->lo[d]) / g->n[d] : 1.0;
    c->bc[d][0] = d < g->dim ? g->bc[d][0] : RT_BC_PERIODIC;
    c->bc[d][1] = d < g->dim ? g->bc[d][1] : RT_BC_PERIODIC;
  }
  c->N = N;
  c->M = M;
  c->C = Crat;
  c->P = Prat;
  c->opt = o;
  c->stream = (cudaStream_t)o.stream;
  c->fp64 = o.precision == RT_FP64;
  c->bf16 = o.precision == RT_BF16;
  c->quad = o.precision == RT_FP32;
  c->rs = c->fp64 ? 8 : 4;
  c->rsI = c->bf16 ? 2 : c->rs;
  c->I_bytes = c->rsI * (size_t)N * (c->quad ? 4 * (size_t)((M + 3) / 4) : (size_t)M);
  c->host_n.assign(ang->n, ang->n + 3 * M);
  c->host_w.assign(ang->w, ang->w + M);
  c->host_inflow.assign(6 * (size_t)M, 0.0);
  c->host_angf.resize(4 * (size_t)M);
  for (int m = 0; m < M; ++m) {
    for (int d = 0; d < 3; ++d) c->host_angf[4 * m + d] = (float)ang->n[3 * m + d];
    c->host_angf[4 * m + 3] = (float)ang->w[m];
  }
  c->host_inflowf.assign(6 * (size_t)M, 0.0f);
  bool ok = c->fp64 ? rtg::choose_tile<double>(c->dim, M, true, &c->tile)
            : c->bf16 ? rtg::choose_tile_b16(c->dim, M, &c->tile)
                      : rtg::choose_tile<float>(c->dim, M, true, &c->tile);
  if (!ok) {
    delete c;
    return fail(RT_E_INVALID, "rt_create: too many angles for one CTA's shared memory");
  }
  size_t rs = c->rs;
  c->stage_len = std::max<long long>(10 * N, (long long)8 * M);
  const size_t Nz = (size_t)N, Mz = (size_t)M;
  struct {
    void **p;
    size_t bytes;
  } allocs[] = {
      {&c->I[0], c->I_bytes},        {&c->I[1], c->I_bytes},        {(void **)&c->mom[0], 8 * 10 * Nz},
      {(void **)&c->mom[1], 8 * 10 * Nz}, {&c->rho, rs * Nz},       {&c->sa, rs * Nz},
      {&c->ss, rs * Nz},         {&c->v, rs * 3 * Nz},             {(void **)&c->T, 8 * Nz},
      {(void **)&c->dEgas, 8 * Nz}, {(void **)&c->dMom, 8 * 3 * Nz}, {&c->ang, rs * 4 * Mz},
      {&c->inflow, rs * 6 * Mz}, {(void **)&c->flags, 2 * sizeof(int)},
      {(void **)&c->stage, sizeof(double) * (size_t)c->stage_len},
      {(void **)&c->qscr, c->bf16 ? sizeof(float) * Mz * Nz : 0},
      {(void **)&c->cen[0], c->quad ? sizeof(float) * Nz : 0},
      {(void **)&c->cen[1], c->quad ? sizeof(float) * Nz : 0},
  };
  for (auto &a : allocs) {
    if (a.bytes == 0) continue;
    if (rtg::device_alloc(a.p, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      free_all(c);
      delete c;
      return fail(RT_E_NOMEM, "rt_create: device allocation failed");
    }
  }
  // angle table [M][4] = (n_x, n_y, n_z, W) and zero inflow, via the stage
  std::vector<double> tab(4 * (size_t)M);
  for (int m = 0; m < M; ++m) {
    for (int d = 0; d < 3; ++d) tab[4 * m + d] = ang->n[3 * m + d];
    tab[4 * m + 3] = ang->w[m];
  }
  rt_status st = RT_OK;
  cudaError_t e = cudaMemcpyAsync(c->stage, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) st = convert_in(c, c->stage, c->ang, 4 * M);
  if (e == cudaSuccess && st == RT_OK) e = cudaMemsetAsync(c->inflow, 0, rs * 6 * M, c->stream);
  if (e == cudaSuccess && st == RT_OK) e = cudaMemsetAsync(c->flags, 0, 2 * sizeof(int), c->stream);
  if (e == cudaSuccess && st == RT_OK) e = cudaMemsetAsync(c->dEgas, 0, 8 * N, c->stream);
  if (e == cudaSuccess && st == RT_OK) e = cudaMemsetAsync(c->dMom, 0, 8 * 3 * N, c->stream);
  if (e == cudaSuccess && st == RT_OK) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess || st != RT_OK) {
    free_all(c);
    delete c;
    return e != cudaSuccess ? cuda_fail(e, "rt_create") : st;
  }
  *out = c;
  return RT_OK;
}

rt_status rt_set_material(rt_ctx *c, const double *rho, const double *T, const double *v, const double *sa,
                          const double *ss) {
  rtg::Range nvtx_range("rt_set_material");
  if (!c || !rho || !T || !v || !sa || !ss) return fail(RT_E_INVALID, "rt_set_material: NULL argument");
  const long long N = c->N;
  if (c->stage_len < 7 * N) return fail(RT_E_STATE, "rt_set_material: staging buffer too small");
  double *s_rho = c->stage, *s_T = c->stage + N, *s_v = c->stage + 2 * N, *s_sa = c->stage + 5 * N,
         *s_ss = c->stage + 6 * N;
  rt_status st;
  if ((st = fetch(c, rho, s_rho, N)) != RT_OK) return st;
  if ((st = fetch(c, T, s_T, N)) != RT_OK) return st;
  if ((st = fetch(c, v, s_v, 3 * N)) != RT_OK) return st;
  if ((st = fetch(c, sa, s_sa, N)) != RT_OK) return st;
  if ((st = fetch(c, ss, s_ss, N)) != RT_OK) return st;
  // scan: bit 0 = a value out of range or non-finite, bit 1 = some v != 0
  RT_CUDA(cudaMemsetAsync(c->flags + 1, 0, sizeof(int), c->stream));
  if ((st = fields_in(c, 0, N, false, c->stream)) != RT_OK) return st;
  int flag = 0;
  RT_CUDA(cudaMemcpyAsync(&flag, c->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  RT_CUDA(cudaStreamSynchronize(c->stream));
  if (flag & 1) return fail(RT_E_NONFINITE, "rt_set_material: need finite rho > 0, T > 0, sigma >= 0, v");
  if ((st = fields_in(c, 0, N, true, c->stream)) != RT_OK) return st;
  const bool vel_before = rtg::velocity_on(c);
  c->has_v = (flag & 2) != 0;
  // a batch compiles its launch for the velocity terms or without them
  if (c->batch && rtg::velocity_on(c) != vel_before) rtg::batch_touch(c->batch);
  c->material_set = true;
  if (!c->intensity_set) return rt_set_intensity(c, nullptr);
  return RT_OK;
}

rt_status rt_set_intensity(rt_ctx *c, const double *I) {
  rtg::Range nvtx_range("rt_set_intensity");
  if (!c) return fail(RT_E_INVALID, "rt_set_intensity: NULL context");
  const long long N = c->N;
  // bf16 storage: the float field goes to the Q scratch first; its moments
  // set J for the encoding below
  void *dst = c->bf16 ? (void *)c->qscr : c->I[c->cur];
  const size_t rsd = c->bf16 ? sizeof(float) : c->rs;
  if (!I) {
    if (!c->material_set) return fail(RT_E_STATE, "rt_set_intensity(NULL) needs rt_set_material first");
    cudaError_t e = c->fp64 ? rtg::launch_isotropic<double>(c->T, (double *)dst, c->M, N, false, c->stream)
                            : rtg::launch_isotropic<float>(c->T, (float *)dst, c->M, N, c->quad, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "isotropic");
  } else {
    // check everything first (finite, >= 0), then convert chunk by chunk
    long long chunk = c->stage_len;
    RT_CUDA(cudaMemsetAsync(c->flags + 1, 0, sizeof(int), c->stream));
    for (long long off = 0; off < (long long)c->M * N; off += chunk) {
      long long n = std::min(chunk, (long long)c->M * N - off);
      rt_status st = fetch(c, I + off, c->stage, n);
      if (st != RT_OK) return st;
      RT_CUDA(rtg::launch_check(c->stage, n, 0.0, 0, 0, c->flags + 1, c->stream));
    }
    int flag = 0;
    RT_CUDA(cudaMemcpyAsync(&flag, c->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    RT_CUDA(cudaStreamSynchronize(c->stream));
    if (flag & 1) return fail(RT_E_NONFINITE, "rt_set_intensity: need finite I >= 0");
    if (c->quad) RT_CUDA(cudaMemsetAsync(dst, 0, c->I_bytes, c->stream));   // the padding angles
    for (long long off = 0; off < (long long)c->M * N; off += chunk) {
      long long n = std::min(chunk, (long long)c->M * N - off);
      rt_status st = fetch(c, I + off, c->stage, n);
      if (st != RT_OK) return st;
      if (c->quad) {
        RT_CUDA(rtg::launch_quad_in(c->stage, (float *)dst, off, n, N, c->stream));
      } else {
        st = convert_in(c, c->stage, (char *)dst + off * rsd, n);
        if (st != RT_OK) return st;
      }
    }
  }
  rt_status st = recompute_moments(c);
  if (st != RT_OK) return st;
  if (c->bf16)
    RT_CUDA(rtg::launch_encode_b16(c->qscr, c->mom[c->cur], (unsigned short *)c->I[c->cur], c->M, N, c->stream));
  // a host array may be page-locked, and then the copies above read it
  // asynchronously: the call returns once they are done
  if (I && !c->opt.device_ptrs) RT_CUDA(cudaStreamSynchronize(c->stream));
  c->intensity_set = true;
  return RT_OK;
}

rt_status rt_set_inflow(rt_ctx *c, int axis, int side, const double *I_ghost) {
  if (!c || !I_ghost) return fail(RT_E_INVALID, "rt_set_inflow: NULL argument");
  if (axis < 0 || axis >= c->dim || side < 0 || side > 1) return fail(RT_E_INVALID, "rt_set_inflow: bad face");
  for (int m = 0; m < c->M; ++m)
    if (!std::isfinite(I_ghost[m]) || I_ghost[m] < 0) return fail(RT_E_NONFINITE, "rt_set_inflow: need finite I >= 0");
  std::copy(I_ghost, I_ghost + c->M, c->host_inflow.begin() + (size_t)(axis * 2 + side) * c->M);
  for (int m = 0; m < c->M; ++m) c->host_inflowf[(size_t)(axis * 2 + side) * c->M + m] = (float)I_ghost[m];
  RT_CUDA(cudaMemcpyAsync(c->stage, c->host_inflow.data(), 6 * c->M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  rt_status st = convert_in(c, c->stage, c->inflow, 6 * c->M);
  if (st != RT_OK) return st;
  RT_CUDA(cudaStreamSynchronize(c->stream));
  // the float step carries the table in its launch parameters: a graph
  // captured by rt_run holds the old one
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return RT_OK;
}

rt_status rt_set_tile(rt_ctx *c, int tx, int ty, int tz) {
  if (!c) return fail(RT_E_INVALID, "rt_set_tile: NULL context");
  rtg::TileShape t{tx, ty, tz};
  if (tx == 0 && ty == 0 && tz == 0) {
    bool ok = c->fp64 ? rtg::choose_tile<double>(c->dim, c->M, true, &t)
              : c->bf16 ? rtg::choose_tile_b16(c->dim, c->M, &t)
                        : rtg::choose_tile<float>(c->dim, c->M, true, &t);
    if (!ok) return fail(RT_E_INVALID, "rt_set_tile: no default tile fits");
  } else {
    bool ok;
    if (c->bf16) {
      rtg::TileShape d;
      ok = rtg::choose_tile_b16(c->dim, c->M, &d) && d.tx == t.tx && d.ty == t.ty && d.tz == t.tz;
    } else {
      ok = c->fp64 ? rtg::tile_ok<double>(c->dim, c->M, true, t) : rtg::tile_ok<float>(c->dim, c->M, true, t);
    }
    if (!ok) return fail(RT_E_INVALID, "rt_set_tile: shape exceeds the thread, shared-memory or staging limits");
  }
  c->tile = t;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return RT_OK;
}

rt_status rt_autotune(rt_ctx *c, int trial_steps, rt_tile_time *times, int cap, int *ntimes) {
  rtg::Range nvtx_range("rt_autotune");
  if (!c) return fail(RT_E_INVALID, "rt_autotune: NULL context");
  if (trial_steps < 1) return fail(RT_E_INVALID, "rt_autotune: trial_steps < 1");
  if (cap < 0 || (cap > 0 && !times)) return fail(RT_E_INVALID, "rt_autotune: bad times buffer");
  if (!c->material_set || !c->intensity_set) return fail(RT_E_STATE, "rt_autotune: set material and intensity first");
  if (c->batch) return fail(RT_E_STATE, "rt_autotune: the context belongs to a batch; use rt_batch_autotune");
  const bool vel = rtg::velocity_on(c);
  rtg::TileShape cand[16];
  int nc = c->fp64 ? rtg::tile_candidates<double>(c->dim, c->M, true, cand)
                   : rtg::tile_candidates<float>(c->dim, c->M, true, cand);
  if (c->bf16) nc = rtg::choose_tile_b16(c->dim, c->M, &cand[0]) ? 1 : 0;   // one compiled tile
  if (nc == 0) return fail(RT_E_INVALID, "rt_autotune: no compiled tile fits");
  // The trial steps read I[cur] and write only I[1 - cur], mom[1 - cur]
  // (scratch until the next real step), T in place and the step sources:
  // save those three and the Newton-failure word, restore them afterwards.
  const size_t N = (size_t)c->N;
  double *save_T = c->stage, *save_dE = c->stage + N, *save_dM = c->stage + 2 * N;
  int flag0 = 0;
  RT_CUDA(cudaMemcpyAsync(&flag0, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  RT_CUDA(cudaMemcpyAsync(save_T, c->T, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  RT_CUDA(cudaMemcpyAsync(save_dE, c->dEgas, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  RT_CUDA(cudaMemcpyAsync(save_dM, c->dMom, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  const double dt = rt_cfl_dt(c);
  cudaEvent_t e0, e1;
  RT_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(RT_E_CUDA, "rt_autotune: event");
  }
  const rtg::TileShape keep = c->tile;
  rtg::TileShape best = keep;
  double best_ms = 0;
  cudaError_t e = cudaSuccess;
  int n_out = 0;
  for (int i = 0; i < nc && e == cudaSuccess; ++i) {
    float ms = 0;
    for (int k = 0; k <= trial_steps && e == cudaSuccess; ++k) {
      if (k == 1) e = cudaEventRecord(e0, c->stream);
      if (e == cudaSuccess)
        e = c->fp64 ? rtg::launch_ctx_step(c, rtg::make_args<double>(c, dt), vel, cand[i])
                    : rtg::launch_ctx_step(c, rtg::make_args<float>(c, dt), vel, cand[i]);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    const double per = (double)ms / trial_steps;
    if (n_out < cap) times[n_out++] = rt_tile_time{cand[i].tx, cand[i].ty, cand[i].tz, per};
    if (i == 0 || per < best_ms) {
      best_ms = per;
      best = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "rt_autotune: trial steps");
  RT_CUDA(cudaMemcpyAsync(c->T, save_T, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  RT_CUDA(cudaMemcpyAsync(c->dEgas, save_dE, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  RT_CUDA(cudaMemcpyAsync(c->dMom, save_dM, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  RT_CUDA(cudaMemcpyAsync(c->flags, &flag0, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  RT_CUDA(cudaStreamSynchronize(c->stream));
  if (ntimes) *ntimes = n_out;
  if (best.tx != keep.tx || best.ty != keep.ty || best.tz != keep.tz) {
    c->tile = best;
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
  }
  return RT_OK;
}

namespace {

struct StateHeader {
  char magic[8];
  int dim, n[3], M, rs, has_v, intensity_set;
  long long N;
  double C, P;
};
const char kStateMagic[8] = {'R', 'T', 'S', 'T', 'A', 'T', 'E', '2'};

// (device pointer, bytes) of every saved array, in file order.
int state_parts(rt_ctx *c, void **ptr, size_t *bytes) {
  const size_t N = (size_t)c->N, M = (size_t)c->M, rs = c->rs;
  int k = 0;
  auto add = [&](void *p, size_t b) { ptr[k] = p; bytes[k] = b; ++k; };
  add(c->I[c->cur], c->I_bytes);
  add(c->mom[c->cur], 8 * 10 * N);
  add(c->T, 8 * N);
  add(c->rho, rs * N);
  add(c->sa, rs * N);
  add(c->ss, rs * N);
  add(c->v, rs * 3 * N);
  add(c->dEgas, 8 * N);
  add(c->dMom, 8 * 3 * N);
  add(c->inflow, rs * 6 * M);
  return k;
}

}  // namespace

size_t rt_state_bytes(const rt_ctx *c) {
  if (!c) return 0;
  void *p[16];
  size_t b[16], total = sizeof(StateHeader) + sizeof(double) * 6 * (size_t)c->M;
  const int k = state_parts(const_cast<rt_ctx *>(c), p, b);
  for (int i = 0; i < k; ++i) total += b[i];
  return total;
}

rt_status rt_save_state(rt_ctx *c, void *buf, size_t bytes) {
  rtg::Range nvtx_range("rt_save_state");
  if (!c || !buf) return fail(RT_E_INVALID, "rt_save_state: NULL argument");
  if (bytes < rt_state_bytes(c)) return fail(RT_E_INVALID, "rt_save_state: buffer smaller than rt_state_bytes");
  if (!c->material_set) return fail(RT_E_STATE, "rt_save_state: call rt_set_material first");
  RT_CUDA(cudaStreamSynchronize(c->stream));
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, 8);
  h.dim = c->dim;
  for (int d = 0; d < 3; ++d) h.n[d] = c->n[d];
  h.M = c->M;
  h.rs = (int)c->rsI;   // bytes per stored intensity: tells the three precisions apart
  h.has_v = c->has_v;
  h.intensity_set = c->intensity_set;
  h.N = c->N;
  h.C = c->C;
  h.P = c->P;
  char *out = static_cast<char *>(buf);
  std::memcpy(out, &h, sizeof h);
  out += sizeof h;
  std::memcpy(out, c->host_inflow.data(), sizeof(double) * 6 * (size_t)c->M);
  out += sizeof(double) * 6 * (size_t)c->M;
  void *p[16];
  size_t b[16];
  const int k = state_parts(c, p, b);
  for (int i = 0; i < k; ++i) {
    RT_CUDA(cudaMemcpyAsync(out, p[i], b[i], cudaMemcpyDeviceToHost, c->stream));
    out += b[i];
  }
  RT_CUDA(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_load_state(rt_ctx *c, const void *buf, size_t bytes) {
  rtg::Range nvtx_range("rt_load_state");
  if (!c || !buf) return fail(RT_E_INVALID, "rt_load_state: NULL argument");
  if (c->batch) return fail(RT_E_STATE, "rt_load_state: the context belongs to a batch");
  if (bytes < sizeof(StateHeader)) return fail(RT_E_INVALID, "rt_load_state: buffer too short");
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  bool same = std::memcmp(h.magic, kStateMagic, 8) == 0 && h.dim == c->dim && h.M == c->M &&
              h.rs == (int)c->rsI && h.N == c->N && h.C == c->C && h.P == c->P;
  for (int d = 0; d < 3; ++d) same = same && h.n[d] == c->n[d];
  if (!same) return fail(RT_E_INVALID, "rt_load_state: the state was saved from a different grid, angle set, precision or Crat/Prat");
  if (bytes < rt_state_bytes(c)) return fail(RT_E_INVALID, "rt_load_state: buffer shorter than the saved state");
  RT_CUDA(cudaStreamSynchronize(c->stream));
  c->cur = 0;
  const char *in = static_cast<const char *>(buf) + sizeof h;
  std::memcpy(c->host_inflow.data(), in, sizeof(double) * 6 * (size_t)c->M);
  // the float step takes its inflow from the host's float table (launch
  // parameters), the batch kernel from the device table restored below
  for (size_t i = 0; i < 6 * (size_t)c->M; ++i) c->host_inflowf[i] = (float)c->host_inflow[i];
  in += sizeof(double) * 6 * (size_t)c->M;
  void *p[16];
  size_t b[16];
  const int k = state_parts(c, p, b);
  for (int i = 0; i < k; ++i) {
    RT_CUDA(cudaMemcpyAsync(p[i], in, b[i], cudaMemcpyHostToDevice, c->stream));
    in += b[i];
  }
  RT_CUDA(cudaMemsetAsync(c->flags, 0, 2 * sizeof(int), c->stream));
  // the float step's cell centers are a function of the intensity: formed
  // again rather than saved
  if (c->quad) RT_CUDA(rtg::launch_centers((const float *)c->I[c->cur], c->M, c->N, c->cen[c->cur], c->stream));
  RT_CUDA(cudaStreamSynchronize(c->stream));
  c->has_v = h.has_v != 0;
  c->intensity_set = h.intensity_set != 0;
  c->material_set = true;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return RT_OK;
}

rt_status rt_get_tile(const rt_ctx *c, int *tx, int *ty, int *tz) {
  if (!c || !tx || !ty || !tz) return fail(RT_E_INVALID, "rt_get_tile: NULL argument");
  *tx = c->tile.tx;
  *ty = c->tile.ty;
  *tz = c->tile.tz;
  return RT_OK;
}

double rt_cfl_dt(const rt_ctx *c) {
  if (!c) return 0.0;
  double h = c->dx[0];
  for (int d = 1; d < c->dim; ++d) h = std::min(h, c->dx[d]);
  return c->opt.cfl * h / c->C;
}

rt_status rt_step(rt_ctx *c, double dt) {
  rtg::Range nvtx_range("rt_step");
  if (!c) return fail(RT_E_INVALID, "rt_step: NULL context");
  if (!c->material_set) return fail(RT_E_STATE, "rt_step: call rt_set_material first");
  if (c->batch) return fail(RT_E_STATE, "rt_step: the context belongs to a batch; step it with rt_batch_step");
  if (!(dt > 0)) dt = rt_cfl_dt(c);
  if (!std::isfinite(dt)) return fail(RT_E_INVALID, "rt_step: dt not finite");
  return launch_step(c, dt);
}

rt_status rt_run(rt_ctx *c, double dt, int nsteps) {
  rtg::Range nvtx_range("rt_run");
  if (!c) return fail(RT_E_INVALID, "rt_run: NULL context");
  if (!c->material_set) return fail(RT_E_STATE, "rt_run: call rt_set_material first");
  if (c->batch) return fail(RT_E_STATE, "rt_run: the context belongs to a batch; step it with rt_batch_step");
  if (nsteps < 0) return fail(RT_E_INVALID, "rt_run: nsteps < 0");
  if (nsteps == 0) return RT_OK;
  if (!(dt > 0)) dt = rt_cfl_dt(c);
  if (!std::isfinite(dt)) return fail(RT_E_INVALID, "rt_run: dt not finite");
  if (c->stream == nullptr) {
    // the legacy default stream cannot be captured: plain launches
    for (int k = 0; k < nsteps; ++k) {
      rt_status st = launch_step(c, dt);
      if (st != RT_OK) return st;
    }
    return RT_OK;
  }
  bool vel = rtg::velocity_on(c);
  if (!c->graph || c->graph_dt != dt || c->graph_steps != nsteps || c->graph_cur != c->cur || c->graph_vel != vel) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    int start = c->cur;
    cudaGraph_t graph;
    RT_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    rt_status st = RT_OK;
    for (int k = 0; k < nsteps && st == RT_OK; ++k) st = launch_step(c, dt);
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    c->cur = start;
    if (st != RT_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "rt_run: capture");
    e = cudaGraphInstantiate(&c->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "rt_run: instantiate");
    c->graph_dt = dt;
    c->graph_steps = nsteps;
    c->graph_cur = start;
    c->graph_vel = vel;
  }
  RT_CUDA(cudaGraphLaunch(c->graph, c->stream));
  if (nsteps % 2) c->cur = 1 - c->cur;
  return RT_OK;
}

rt_status rt_sync(rt_ctx *c) {
  if (!c) return fail(RT_E_INVALID, "rt_sync: NULL context");
  int bad = 0;
  RT_CUDA(cudaMemcpyAsync(&bad, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  RT_CUDA(cudaStreamSynchronize(c->stream));
  if (bad) {
    RT_CUDA(cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream));
    RT_CUDA(cudaStreamSynchronize(c->stream));
    char msg[96];
    std::snprintf(msg, sizeof msg, "T^4 Newton iteration failed in %d cell-steps", bad);
    return fail(RT_E_NONFINITE, msg);
  }
  return RT_OK;
}

rt_status rt_moments(rt_ctx *c, double *E, double *F, double *P) {
  rtg::Range nvtx_range("rt_moments");
  if (!c) return fail(RT_E_INVALID, "rt_moments: NULL context");
  if (!c->intensity_set) return fail(RT_E_STATE, "rt_moments: no intensity yet");
  const long long N = c->N;
  const double *mom = c->mom[c->cur];
  rt_status st;
  if (E && (st = deliver_async(c, mom, E, N)) != RT_OK) return st;
  if (F && (st = deliver_async(c, mom + N, F, 3 * N)) != RT_OK) return st;
  if (P && (st = deliver_async(c, mom + 4 * N, P, 6 * N)) != RT_OK) return st;
  return delivered(c);
}

rt_status rt_eddington(rt_ctx *c, double *f) {
  rtg::Range nvtx_range("rt_eddington");
  if (!c || !f) return fail(RT_E_INVALID, "rt_eddington: NULL argument");
  if (!c->intensity_set) return fail(RT_E_STATE, "rt_eddington: no intensity yet");
  const long long N = c->N;
  double *dst = c->opt.device_ptrs ? f : c->stage;
  RT_CUDA(rtg::launch_eddington(c->mom[c->cur], dst, N, c->stream));
  if (c->opt.device_ptrs) return RT_OK;
  return deliver(c, c->stage, f, 6 * N);
}

rt_status rt_sources(rt_ctx *c, double *dE_gas, double *dMom, double *T_new) {
  rtg::Range nvtx_range("rt_sources");
  if (!c) return fail(RT_E_INVALID, "rt_sources: NULL context");
  const long long N = c->N;
  rt_status st;
  // the energy source and T are double on the device: copied out directly
  if (dE_gas && (st = deliver_async(c, c->dEgas, dE_gas, N)) != RT_OK) return st;
  if (dMom && (st = deliver_async(c, c->dMom, dMom, 3 * N)) != RT_OK) return st;
  if (T_new && (st = deliver_async(c, c->T, T_new, N)) != RT_OK) return st;
  return delivered(c);
}

rt_status rt_step_coupled(rt_ctx *c, double dt, const double *rho, const double *T, const double *v,
                          const double *sa, const double *ss, double *dE_gas, double *dMom, double *T_new) {
  rtg::Range nvtx_range("rt_step_coupled");
  if (!c) return fail(RT_E_INVALID, "rt_step_coupled: NULL context");
  if (!rho || !T || !v || !sa || !ss) return fail(RT_E_INVALID, "rt_step_coupled: NULL field");
  if (c->batch) return fail(RT_E_STATE, "rt_step_coupled: the context belongs to a batch");
  // slabs along the outermost active axis (z in 3-D, y in 2-D, x in 1-D);
  // a "plane" is the set of cells with one coordinate along it
  const int d_out = std::max(0, c->dim - 1);
  const int nz = c->n[d_out];
  const int TZ = std::max(1, d_out == 2 ? c->tile.tz : d_out == 1 ? c->tile.ty : c->tile.tx);
  const int layers = (nz + TZ - 1) / TZ;
  if (c->opt.device_ptrs || c->bf16 || !c->material_set || !c->intensity_set || layers < 2 ||
      c->stage_len < 10 * c->N) {
    // the three calls in turn
    rt_status st = rt_set_material(c, rho, T, v, sa, ss);
    if (st == RT_E_NONFINITE) c->material_set = false;
    if (st == RT_OK) st = rt_step(c, dt);
    if (st == RT_OK) st = rt_sources(c, dE_gas, dMom, T_new);
    return st;
  }
  if (!(dt > 0)) dt = rt_cfl_dt(c);
  if (!std::isfinite(dt)) return fail(RT_E_INVALID, "rt_step_coupled: dt not finite");
  rt_status st = coupled_init(c);
  if (st != RT_OK) return st;
  long long Nxy = 1;   // cells per plane
  for (int d = 0; d < d_out; ++d) Nxy *= c->n[d];
  const int S = std::min(rt_ctx::kSlabs, layers);
  int L[rt_ctx::kSlabs + 1], e[rt_ctx::kSlabs];   // slab s: tile layers [L[s], L[s+1]), planes up to e[s]
  // Slab sizes double from each end towards the middle (weights 1, 2, 4,
  // ..., 4, 2, 1): nothing overlaps the first slab's fields going over or
  // the last slab's sources coming back, so both are one layer; every other
  // slab's fields arrive while the slab before it runs (the link moves a
  // layer's fields ~3x faster than the kernel steps it), and its sources go
  // back while the slabs after it run.
  {
    double w[rt_ctx::kSlabs], wsum = 0, acc = 0;
    for (int s = 0; s < S; ++s) wsum += (w[s] = std::ldexp(1.0, std::min(s, S - 1 - s)));
    L[0] = 0;
    for (int s = 0; s < S; ++s) {
      acc += w[s];
      L[s + 1] = std::max(L[s] + 1, (int)std::llround(layers * acc / wsum));
    }
    L[S] = layers;
    for (int s = S - 1; s >= 1; --s) L[s] = std::min(L[s], L[s + 1] - 1);
  }
  for (int s = 0; s < S; ++s) e[s] = std::min(L[s + 1] * TZ, nz);
  // A slab reads the fields of two planes beyond its own on each side.  The
  // planes go over in order, each once: slab s needs those below
  // min(top, e[s] + 2), and the top planes [top, nz) go first, for slab 0's
  // periodic wrap.
  const int top = std::min(nz, std::max(nz - 2, e[0] + 2));
  const double *f[5] = {rho, T, v, sa, ss};
  // the Newton-failure count of earlier steps, restored if the fields fail
  // (cells stepped with bad fields must not count against the next rt_sync)
  int failures = 0;
  RT_CUDA(cudaMemcpyAsync(&failures, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  RT_CUDA(cudaMemsetAsync(c->flags + 1, 0, sizeof(int), c->stream));
  // the staging buffer, the outputs and the scan flag are free once the
  // context's stream reaches this point
  RT_CUDA(cudaEventRecord(c->ev_start, c->stream));
  RT_CUDA(cudaStreamWaitEvent(c->xs_in, c->ev_start, 0));
  RT_CUDA(cudaStreamWaitEvent(c->xs_cv, c->ev_start, 0));
  RT_CUDA(cudaStreamWaitEvent(c->xs_out, c->ev_start, 0));
  RT_CUDA(cudaStreamWaitEvent(c->xs_k, c->ev_start, 0));
  const bool vel = rtg::velocity_on(c);   // kernel of the previous fields; checked below
  int sent = 0;
  for (int s = 0; s < S; ++s) {
    const int upto = std::min(top, e[s] + 2);
    if (s == 0 && top < nz && (st = coupled_in(c, f, top * Nxy, nz * Nxy)) != RT_OK) return st;
    if (upto > sent && (st = coupled_in(c, f, sent * Nxy, upto * Nxy)) != RT_OK) return st;
    // scan and convert on their own stream as the planes arrive, so that a
    // chunk's conversion can run in the tail of the previous slab
    RT_CUDA(cudaEventRecord(c->ev_copied[s], c->xs_in));
    RT_CUDA(cudaStreamWaitEvent(c->xs_cv, c->ev_copied[s], 0));
    if (s == 0 && top < nz && (st = fields_in(c, top * Nxy, nz * Nxy, true, c->xs_cv)) != RT_OK) return st;
    if (upto > sent && (st = fields_in(c, sent * Nxy, upto * Nxy, true, c->xs_cv)) != RT_OK) return st;
    RT_CUDA(cudaEventRecord(c->ev_in[s], c->xs_cv));
    // slabs alternate between two streams, so that a slab's first CTAs take
    // the SMs that the previous slab's last wave leaves idle (the slabs
    // write disjoint cells and read only step-n state and converted fields)
    cudaStream_t ks = (s & 1) ? c->xs_k : c->stream;
    RT_CUDA(cudaStreamWaitEvent(ks, c->ev_in[s], 0));
    sent = std::max(sent, upto);
    if ((st = coupled_launch(c, dt, vel, L[s], L[s + 1], ks)) != RT_OK) return st;
    const long long c0 = (long long)L[s] * TZ * Nxy, c1 = (long long)e[s] * Nxy;
    if ((st = coupled_out(c, c0, c1, c->ev_done[s], ks, dE_gas, dMom, T_new)) != RT_OK) return st;
  }
  if (S > 1) {
    // the context's stream goes on after the last slab of the second stream
    const int last_k = ((S - 1) & 1) ? S - 1 : S - 2;
    RT_CUDA(cudaStreamWaitEvent(c->stream, c->ev_done[last_k], 0));
  }
  int flag = 0;
  RT_CUDA(cudaMemcpyAsync(&flag, c->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  RT_CUDA(cudaStreamSynchronize(c->stream));
  RT_CUDA(cudaStreamSynchronize(c->xs_out));
  if (flag & 1) {
    // T was stepped in place and the fields are partly new: neither is usable
    c->material_set = false;
    RT_CUDA(cudaMemcpy(c->flags, &failures, sizeof(int), cudaMemcpyHostToDevice));
    return fail(RT_E_NONFINITE, "rt_step_coupled: need finite rho > 0, T > 0, sigma >= 0, v");
  }
  c->has_v = (flag & 2) != 0;
  if (rtg::velocity_on(c) != vel) {
    // the fields switched the velocity terms on or off: step again from the
    // staged T with the other kernel
    RT_CUDA(cudaMemcpyAsync(c->T, c->stage + c->N, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if ((st = coupled_launch(c, dt, !vel, 0, 0, c->stream)) != RT_OK) return st;
    c->cur = 1 - c->cur;
    return rt_sources(c, dE_gas, dMom, T_new);
  }
  c->cur = 1 - c->cur;
  return RT_OK;
}

rt_status rt_get_intensity(rt_ctx *c, double *I) {
  rtg::Range nvtx_range("rt_get_intensity");
  if (!c || !I) return fail(RT_E_INVALID, "rt_get_intensity: NULL argument");
  if (!c->intensity_set) return fail(RT_E_STATE, "rt_get_intensity: no intensity yet");
  long long total = (long long)c->M * c->N, chunk = c->stage_len;
  for (long long off = 0; off < total; off += chunk) {
    long long n = std::min(chunk, total - off);
    rt_status st = RT_OK;
    if (c->bf16) {
      cudaError_t e = rtg::launch_decode_b16((const unsigned short *)c->I[c->cur], c->mom[c->cur], c->stage, off, n,
                                             c->N, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "decode");
    } else if (c->quad) {
      cudaError_t e = rtg::launch_quad_out((const float *)c->I[c->cur], c->stage, off, n, c->N, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "quad layout");
    } else {
      st = convert_out(c, (const char *)c->I[c->cur] + off * c->rs, c->stage, n);
    }
    if (st != RT_OK) return st;
    if ((st = deliver(c, c->stage, I + off, n)) != RT_OK) return st;
  }
  return RT_OK;
}

void rt_destroy(rt_ctx *c) {
  if (!c) return;
  if (c->batch) rt_batch_remove((rt_batch *)c->batch, c);
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

}  // extern "C"
