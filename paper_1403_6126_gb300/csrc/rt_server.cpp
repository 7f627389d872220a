// Serving loop: continuous batching of transfer solves.
//
// rt_submit copies a request (grid, angles, gas fields, step count) into the
// server and returns a ticket.  A server thread admits queued requests in
// arrival order whenever the HBM budget has room (first fit: a request that
// does not fit yet does not block smaller ones behind it), creates their
// device state, and adds them to one batch; every loop iteration advances all
// live problems by one step with one persistent launch, so requests that
// arrive while others run join at the next step boundary and share the
// device.  A problem that has done its steps has its moments copied to host
// memory, its device state freed and its ticket marked done; rt_poll hands
// the result over.  Latency is measured from rt_submit to the moment the
// result is in host memory.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rt.h"
#include "rt_ctx.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  rt_ticket id = 0;
  rt_grid grid{};
  std::vector<double> n, w, rho, T, v, sa, ss;
  std::vector<double> inflow;   // [3][2][M] for RT_BC_INFLOW faces, or empty
  double C = 1, P = 1;
  int nsteps = 0, done_steps = 0;
  size_t bytes = 0;
  long long N = 0;
  rt_ctx *ctx = nullptr;
  enum { QUEUED, RUNNING, DONE } state = QUEUED;
  rt_status status = RT_OK;
  std::string error;
  std::vector<double> E, F, Pm;
  double t_submit = 0, t_done = 0;
};

}  // namespace

struct rt_server {
  size_t budget = 0, used = 0;
  rt_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::deque<Request *> queue;
  std::vector<Request *> live;
  std::unordered_map<rt_ticket, Request *> all;
  rt_batch *batch = nullptr;
  std::thread th;
  bool stop = false;
  rt_ticket next_id = 1;
  long long steps = 0;
};

namespace {

void finish(rt_server *s, Request *r, rt_status st, const std::string &err) {
  if (r->ctx) {
    if (st == RT_OK) {
      st = rt_sync(r->ctx);
      if (st == RT_OK) {
        r->E.resize(r->N);
        r->F.resize(3 * r->N);
        r->Pm.resize(6 * r->N);
        st = rt_moments(r->ctx, r->E.data(), r->F.data(), r->Pm.data());
      }
    }
    std::string msg = st == RT_OK ? err : std::string(rt_last_error());
    rt_batch_remove(s->batch, r->ctx);
    rt_destroy(r->ctx);
    r->ctx = nullptr;
    r->error = msg;
  } else {
    r->error = err;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  s->used -= r->bytes;
  r->status = st;
  r->t_done = now_s();
  r->state = Request::DONE;
  s->live.erase(std::remove(s->live.begin(), s->live.end(), r), s->live.end());
  s->done_cv.notify_all();
}

rt_status start(rt_server *s, Request *r) {
  rt_angles a{(int)r->w.size(), r->n.data(), r->w.data()};
  rt_options o = s->opt;
  o.stream = s->stream;
  o.device_ptrs = 0;
  o.precision = RT_FP32;
  rt_status st = rt_create(&r->grid, &a, r->C, r->P, &o, &r->ctx);
  if (st != RT_OK) return st;
  const int M = (int)r->w.size();
  for (int d = 0; d < r->grid.dim && !r->inflow.empty(); ++d)
    for (int side = 0; side < 2; ++side)
      if (r->grid.bc[d][side] == RT_BC_INFLOW) {
        st = rt_set_inflow(r->ctx, d, side, r->inflow.data() + (size_t)(d * 2 + side) * M);
        if (st != RT_OK) return st;
      }
  st = rt_set_material(r->ctx, r->rho.data(), r->T.data(), r->v.data(), r->sa.data(), r->ss.data());
  if (st != RT_OK) return st;
  // host copies are no longer needed once the state is on the device
  std::vector<double>().swap(r->rho);
  std::vector<double>().swap(r->T);
  std::vector<double>().swap(r->v);
  std::vector<double>().swap(r->sa);
  std::vector<double>().swap(r->ss);
  return rt_batch_add(s->batch, r->ctx);
}

void loop(rt_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request *> admit;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->work_cv.wait(lock, [&] { return s->stop || !s->queue.empty() || !s->live.empty(); });
      if (s->stop) break;
      for (auto it = s->queue.begin(); it != s->queue.end();) {
        if (s->used + (*it)->bytes <= s->budget) {
          s->used += (*it)->bytes;
          (*it)->state = Request::RUNNING;
          s->live.push_back(*it);
          admit.push_back(*it);
          it = s->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    for (Request *r : admit) {
      rt_status st = start(s, r);
      if (st != RT_OK) finish(s, r, st, rt_last_error());
    }
    std::vector<Request *> live;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      live = s->live;
    }
    if (live.empty()) continue;
    rtg::Range nvtx_range("rt_server step");
    rt_status st = rt_batch_step(s->batch, 1);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    s->steps += 1;
    for (Request *r : live) {
      if (st != RT_OK || e != cudaSuccess) {
        finish(s, r, st != RT_OK ? st : RT_E_CUDA, st != RT_OK ? rt_last_error() : cudaGetErrorString(e));
        continue;
      }
      if (++r->done_steps >= r->nsteps) finish(s, r, RT_OK, "");
    }
  }
}

rt_status fail(rt_status st, const std::string &m) { return rtg::set_error(st, m); }

// Servers still alive when the process exits are stopped first: their
// threads must not run into the CUDA runtime's own teardown.  The handler
// is registered after the runtime has initialised (rt_server_create makes a
// CUDA call first), so it runs before the runtime's.
std::mutex g_live_mu;
std::vector<rt_server *> g_live;

void stop_live_servers() {
  std::vector<rt_server *> live;
  {
    std::lock_guard<std::mutex> lock(g_live_mu);
    live.swap(g_live);
  }
  for (rt_server *s : live) rt_server_destroy(s);
}

void track(rt_server *s) {
  static const bool registered = (std::atexit(stop_live_servers), true);
  (void)registered;
  std::lock_guard<std::mutex> lock(g_live_mu);
  g_live.push_back(s);
}

void untrack(rt_server *s) {
  std::lock_guard<std::mutex> lock(g_live_mu);
  g_live.erase(std::remove(g_live.begin(), g_live.end(), s), g_live.end());
}

}  // namespace

extern "C" {

rt_status rt_server_create(size_t hbm_budget_bytes, const rt_options *opts, rt_server **out) {
  if (!out) return fail(RT_E_INVALID, "rt_server_create: out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0) return fail(RT_E_INVALID, "rt_server_create: zero budget");
  rt_server *s = new (std::nothrow) rt_server;
  if (!s) return fail(RT_E_NOMEM, "rt_server_create: host allocation");
  rt_options_default(&s->opt);
  if (opts) s->opt = *opts;
  if (rt_status st = rtg::check_newton_options(s->opt, "rt_server_create"); st != RT_OK) {
    delete s;
    return st;
  }
  s->budget = hbm_budget_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    return fail(RT_E_CUDA, std::string("rt_server_create: ") + cudaGetErrorString(e));
  }
  rt_status st = rt_batch_create(s->stream, &s->batch);
  if (st != RT_OK) {
    cudaStreamDestroy(s->stream);
    delete s;
    return st;
  }
  s->th = std::thread(loop, s);
  track(s);
  *out = s;
  return RT_OK;
}

rt_status rt_submit(rt_server *s, const rt_grid *g, const rt_angles *a, double Crat, double Prat, const double *rho,
                    const double *T, const double *v, const double *sa, const double *ss, int nsteps,
                    rt_ticket *out) {
  return rt_submit_inflow(s, g, a, Crat, Prat, rho, T, v, sa, ss, nullptr, nsteps, out);
}

rt_status rt_submit_inflow(rt_server *s, const rt_grid *g, const rt_angles *a, double Crat, double Prat,
                           const double *rho, const double *T, const double *v, const double *sa, const double *ss,
                           const double *inflow, int nsteps, rt_ticket *out) {
  rtg::Range nvtx_range("rt_submit");
  if (!s || !g || !a || !a->n || !a->w || !rho || !T || !v || !sa || !ss || !out)
    return fail(RT_E_INVALID, "rt_submit: NULL argument");
  if (nsteps < 1) return fail(RT_E_INVALID, "rt_submit: nsteps < 1");
  if (g->dim < 1 || g->dim > 3) return fail(RT_E_INVALID, "rt_submit: dim must be 1, 2 or 3");
  long long N = 1;
  for (int d = 0; d < g->dim; ++d) {
    if (g->n[d] < 1) return fail(RT_E_INVALID, "rt_submit: empty axis");
    N *= g->n[d];
  }
  if (N >= (1LL << 28)) return fail(RT_E_INVALID, "rt_submit: more than 2^28 cells");
  if (a->m < 1 || a->m > 256) return fail(RT_E_INVALID, "rt_submit: angle count outside 1..256");
  bool vel = s->opt.estimate_v != 0;
  for (long long i = 0; i < 3 * N && !vel; ++i) vel = v[i] != 0.0;
  if (!rtg::batch_fits(g->dim, a->m, vel))
    return fail(RT_E_INVALID, "rt_submit: too many angles for the batch tile's shared memory");
  if (inflow)
    for (long long i = 0; i < 6LL * a->m; ++i)
      if (!std::isfinite(inflow[i]) || inflow[i] < 0) return fail(RT_E_NONFINITE, "rt_submit: need finite inflow I >= 0");
  Request *r = new (std::nothrow) Request;
  if (!r) return fail(RT_E_NOMEM, "rt_submit: host allocation");
  r->grid = *g;
  r->n.assign(a->n, a->n + 3 * a->m);
  r->w.assign(a->w, a->w + a->m);
  r->C = Crat;
  r->P = Prat;
  r->N = N;
  r->rho.assign(rho, rho + N);
  r->T.assign(T, T + N);
  r->v.assign(v, v + 3 * N);
  r->sa.assign(sa, sa + N);
  r->ss.assign(ss, ss + N);
  if (inflow) r->inflow.assign(inflow, inflow + 6 * a->m);
  r->nsteps = nsteps;
  r->bytes = rtg::context_bytes(N, a->m, false);
  if (r->bytes > s->budget) {
    delete r;
    return fail(RT_E_BUDGET, "rt_submit: the problem alone exceeds the HBM budget");
  }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->queue.push_back(r);
  }
  s->work_cv.notify_one();
  *out = r->id;
  return RT_OK;
}

rt_status rt_poll(rt_server *s, rt_ticket t, double *E, double *F, double *P, double *latency_s) {
  if (!s) return fail(RT_E_INVALID, "rt_poll: NULL server");
  Request *r = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(t);
    if (it == s->all.end()) return fail(RT_E_INVALID, "rt_poll: unknown or already collected ticket");
    r = it->second;
    if (r->state != Request::DONE) return RT_PENDING;
    s->all.erase(it);
  }
  rt_status st = r->status;
  if (st == RT_OK) {
    if (E) std::memcpy(E, r->E.data(), sizeof(double) * r->N);
    if (F) std::memcpy(F, r->F.data(), sizeof(double) * 3 * r->N);
    if (P) std::memcpy(P, r->Pm.data(), sizeof(double) * 6 * r->N);
    if (latency_s) *latency_s = r->t_done - r->t_submit;
  } else {
    fail(st, "rt_poll: " + r->error);
  }
  delete r;
  return st;
}

rt_status rt_server_wait(rt_server *s, rt_ticket t, double timeout_s) {
  if (!s) return fail(RT_E_INVALID, "rt_server_wait: NULL server");
  if (std::isnan(timeout_s)) return fail(RT_E_INVALID, "rt_server_wait: timeout is NaN");
  std::unique_lock<std::mutex> lock(s->mu);
  if (s->all.find(t) == s->all.end())
    return fail(RT_E_INVALID, "rt_server_wait: unknown or already collected ticket");
  // The request is looked up again at every wake-up: another thread may
  // collect it with rt_poll meanwhile, which frees it (rt_poll collects only
  // finished requests, so a ticket gone from the table is done).
  auto pred = [&] {
    auto it = s->all.find(t);
    return it == s->all.end() || it->second->state == Request::DONE;
  };
  // beyond about ten years the limit is no limit (and the conversion to the
  // clock's integer ticks cannot overflow)
  if (timeout_s < 0 || timeout_s > 3e8) {
    s->done_cv.wait(lock, pred);
  } else if (!s->done_cv.wait_for(lock, std::chrono::duration<double>(timeout_s), pred)) {
    return fail(RT_E_TIMEOUT, "rt_server_wait: timed out");
  }
  return RT_OK;
}

rt_status rt_server_stats(rt_server *s, long long *steps, int *queued, int *running, size_t *bytes_in_use) {
  if (!s) return fail(RT_E_INVALID, "rt_server_stats: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (steps) *steps = s->steps;
  if (queued) *queued = (int)s->queue.size();
  if (running) *running = (int)s->live.size();
  if (bytes_in_use) *bytes_in_use = s->used;
  return RT_OK;
}

void rt_server_destroy(rt_server *s) {
  if (!s) return;
  untrack(s);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->work_cv.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto &kv : s->all) {
    Request *r = kv.second;
    if (r->ctx) {
      rt_batch_remove(s->batch, r->ctx);
      rt_destroy(r->ctx);
    }
    delete r;
  }
  rt_batch_destroy(s->batch);
  cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
