// Many independent problems advanced by one persistent launch per step.
//
// A batch holds contexts created with rt_create (float intensities).  For a
// step, a device work list names every (problem, tile) pair; a grid of
// persistent CTAs (as many as fit on the GPU at the shared-memory size the
// largest angle set needs) takes items b, b + grid, b + 2 grid, ... and runs
// the same per-tile code as the single-problem kernel, so each problem's
// result is bitwise the one it gets alone.  Items are ordered by decreasing
// angle count, so the long tiles start first and the interleave gives every
// CTA a like share.  Steps are captured in a CUDA graph (one kernel per step)
// and replayed.  Three tile sets are
// compiled (rt_batch_k*.cu); rt_batch_autotune times them on the batch's own
// members and keeps the fastest.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rt.h"
#include "rt_batch_kernel.cuh"
#include "rt_ctx.h"

namespace rtg {

const BatchVariant &batch_variant(int i) {
  static const BatchVariant table[kBatchVariants] = {batch_variant_512(), batch_variant_256(), batch_variant_128()};
  return table[i];
}

static size_t variant_smem(const BatchVariant &v, int dim, int M, bool vel) {
  const TileShape t = dim == 1 ? v.t1 : dim == 2 ? v.t2 : v.t3;
  return stepk::smem_bytes_q(dim, M, vel, t.tx, t.ty, t.tz, false);
}

bool batch_fits(int dim, int M, bool vel) {
  // the default variant's tile must hold the angle set
  return variant_smem(batch_variant(0), dim, M, vel) <= 227 * 1024;
}

}  // namespace rtg

struct rt_batch {
  cudaStream_t stream = nullptr;
  std::vector<rt_ctx *> ctxs;
  bool dirty = true;
  bool vel = false;
  int nitems = 0, grid = 0, phase = 0, variant = 0;
  size_t smem = 0;
  rtg::WorkItem *d_items = nullptr;
  rtg::StepArgs<float> *d_desc[2] = {nullptr, nullptr};
  size_t items_cap = 0, desc_cap = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0, graph_phase = -1;
};

void rtg::batch_touch(void *batch) {
  if (batch) static_cast<rt_batch *>(batch)->dirty = true;
}

namespace {

rt_status cuda_err(cudaError_t e, const char *what) {
  return rtg::set_error(RT_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RT_BCUDA(call)                                   \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_err(_e, #call);   \
  } while (0)

void drop_graph(rt_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

// Rebuilds the work list and both descriptor arrays (current parity of each
// problem and the flipped one) after the membership changed.
rt_status rebuild(rt_batch *b) {
  rtg::Range nvtx_range("rt_batch rebuild");
  drop_graph(b);
  std::vector<int> order(b->ctxs.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->ctxs[x]->M > b->ctxs[y]->M; });
  const rtg::BatchVariant &var = rtg::batch_variant(b->variant);
  std::vector<rtg::WorkItem> items;
  int Mmax = 1;
  bool dims[4] = {false, false, false, false};
  b->vel = false;
  for (rt_ctx *c : b->ctxs) b->vel = b->vel || rtg::velocity_on(c);
  for (int i : order) {
    rt_ctx *c = b->ctxs[i];
    Mmax = std::max(Mmax, c->M);
    dims[c->dim] = true;
    const rtg::TileShape t = c->dim == 1 ? var.t1 : c->dim == 2 ? var.t2 : var.t3;
    const int tx = t.tx, ty = t.ty, tz = t.tz;
    for (int z = 0; z < (c->n[2] + tz - 1) / tz; ++z)
      for (int y = 0; y < (c->n[1] + ty - 1) / ty; ++y)
        for (int x = 0; x < (c->n[0] + tx - 1) / tx; ++x) items.push_back({i, x, y, z});
  }
  size_t smem = 0;
  for (int d = 1; d <= 3; ++d)
    if (dims[d]) smem = std::max(smem, rtg::variant_smem(var, d, Mmax, b->vel));
  if (smem > 227 * 1024)
    return rtg::set_error(RT_E_INVALID, "rt_batch: the largest angle set does not fit the batch tile in shared memory");
  b->smem = smem;
  b->nitems = (int)items.size();
  if (items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;   // consistent if the allocation fails
    RT_BCUDA(rtg::device_alloc((void **)&b->d_items, sizeof(rtg::WorkItem) * items.size()));
    b->items_cap = items.size();
  }
  if (!items.empty())
    RT_BCUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(rtg::WorkItem) * items.size(), cudaMemcpyHostToDevice,
                             b->stream));
  std::vector<rtg::StepArgs<float>> desc[2];
  for (int p = 0; p < 2; ++p) {
    for (rt_ctx *c : b->ctxs) {
      int cur = c->cur;
      c->cur = p ? 1 - cur : cur;
      desc[p].push_back(rtg::make_args<float>(c, rt_cfl_dt(c)));
      c->cur = cur;
    }
  }
  if (b->ctxs.size() > b->desc_cap) {
    b->desc_cap = 0;   // consistent if an allocation fails
    for (int p = 0; p < 2; ++p) {
      if (b->d_desc[p]) cudaFree(b->d_desc[p]);
      b->d_desc[p] = nullptr;
      RT_BCUDA(rtg::device_alloc((void **)&b->d_desc[p], sizeof(rtg::StepArgs<float>) * b->ctxs.size()));
    }
    b->desc_cap = b->ctxs.size();
  }
  for (int p = 0; p < 2; ++p)
    if (!desc[p].empty())
      RT_BCUDA(cudaMemcpyAsync(b->d_desc[p], desc[p].data(), sizeof(rtg::StepArgs<float>) * desc[p].size(),
                               cudaMemcpyHostToDevice, b->stream));
  RT_BCUDA(cudaStreamSynchronize(b->stream));
  int per_sm = 0, dev = 0, sms = 0;
  RT_BCUDA(var.prepare(b->vel, b->smem, &per_sm));
  RT_BCUDA(cudaGetDevice(&dev));
  RT_BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  b->grid = std::max(1, std::min(b->nitems, sms * std::max(1, per_sm)));
  b->phase = 0;
  b->dirty = false;
  return RT_OK;
}

// Queues one step: one persistent launch.
rt_status enqueue_step(rt_batch *b, int parity) {
  RT_BCUDA(rtg::batch_variant(b->variant)
                .launch(b->vel, b->grid, b->smem, b->d_desc[parity], b->d_items, b->nitems, b->stream));
  return RT_OK;
}

}  // namespace

extern "C" {

rt_status rt_batch_create(void *stream, rt_batch **out) {
  if (!out) return rtg::set_error(RT_E_INVALID, "rt_batch_create: out is NULL");
  *out = nullptr;
  rt_batch *b = new (std::nothrow) rt_batch;
  if (!b) return rtg::set_error(RT_E_NOMEM, "rt_batch_create: host allocation");
  b->stream = (cudaStream_t)stream;
  *out = b;
  return RT_OK;
}

rt_status rt_batch_add(rt_batch *b, rt_ctx *c) {
  if (!b || !c) return rtg::set_error(RT_E_INVALID, "rt_batch_add: NULL argument");
  if (c->fp64 || c->bf16) return rtg::set_error(RT_E_INVALID, "rt_batch_add: batches run float intensities (RT_FP32)");
  if (c->stream != b->stream) return rtg::set_error(RT_E_INVALID, "rt_batch_add: context and batch streams differ");
  if (!c->material_set) return rtg::set_error(RT_E_STATE, "rt_batch_add: call rt_set_material first");
  if (std::find(b->ctxs.begin(), b->ctxs.end(), c) != b->ctxs.end())
    return rtg::set_error(RT_E_INVALID, "rt_batch_add: context already in the batch");
  if (c->batch) return rtg::set_error(RT_E_STATE, "rt_batch_add: context already belongs to a batch");
  b->ctxs.push_back(c);
  c->batch = b;
  b->dirty = true;
  return RT_OK;
}

rt_status rt_batch_remove(rt_batch *b, rt_ctx *c) {
  if (!b || !c) return rtg::set_error(RT_E_INVALID, "rt_batch_remove: NULL argument");
  auto it = std::find(b->ctxs.begin(), b->ctxs.end(), c);
  if (it == b->ctxs.end()) return rtg::set_error(RT_E_INVALID, "rt_batch_remove: context not in the batch");
  b->ctxs.erase(it);
  c->batch = nullptr;
  b->dirty = true;
  return RT_OK;
}

int rt_batch_size(const rt_batch *b) { return b ? (int)b->ctxs.size() : 0; }

rt_status rt_batch_step(rt_batch *b, int nsteps) {
  rtg::Range nvtx_range("rt_batch_step");
  if (!b) return rtg::set_error(RT_E_INVALID, "rt_batch_step: NULL batch");
  if (nsteps < 0) return rtg::set_error(RT_E_INVALID, "rt_batch_step: nsteps < 0");
  if (nsteps == 0 || b->ctxs.empty()) return RT_OK;
  if (b->dirty) {
    rt_status st = rebuild(b);
    if (st != RT_OK) return st;
  }
  if (b->stream == nullptr) {
    for (int k = 0; k < nsteps; ++k) {
      rt_status st = enqueue_step(b, (b->phase + k) & 1);
      if (st != RT_OK) return st;
    }
  } else {
    if (!b->graph || b->graph_steps != nsteps || b->graph_phase != b->phase) {
      drop_graph(b);
      cudaGraph_t g;
      RT_BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      rt_status st = RT_OK;
      for (int k = 0; k < nsteps && st == RT_OK; ++k) st = enqueue_step(b, (b->phase + k) & 1);
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (st != RT_OK) return st;
      if (e != cudaSuccess) return cuda_err(e, "rt_batch_step: capture");
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_err(e, "rt_batch_step: instantiate");
      b->graph_steps = nsteps;
      b->graph_phase = b->phase;
    }
    RT_BCUDA(cudaGraphLaunch(b->graph, b->stream));
  }
  if (nsteps & 1)
    for (rt_ctx *c : b->ctxs) c->cur = 1 - c->cur;
  b->phase = (b->phase + nsteps) & 1;
  return RT_OK;
}

rt_status rt_batch_autotune(rt_batch *b, int trial_steps, double *ms, int *chosen) {
  rtg::Range nvtx_range("rt_batch_autotune");
  if (!b) return rtg::set_error(RT_E_INVALID, "rt_batch_autotune: NULL batch");
  if (trial_steps < 1) return rtg::set_error(RT_E_INVALID, "rt_batch_autotune: trial_steps < 1");
  if (b->ctxs.empty()) {
    if (chosen) *chosen = b->variant;
    return RT_OK;
  }
  // Trial launches all use the current parity: they read each member's
  // I[cur] and mom[cur] and write only I[1 - cur] and mom[1 - cur] (scratch
  // until the next real step), T in place and the step sources.  Save those
  // and the Newton-failure words, restore them afterwards.
  std::vector<int> flags(b->ctxs.size(), 0);
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    rt_ctx *c = b->ctxs[i];
    const size_t N = (size_t)c->N;
    RT_BCUDA(cudaMemcpyAsync(c->stage, c->T, N * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    RT_BCUDA(cudaMemcpyAsync(c->stage + N, c->dEgas, N * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    RT_BCUDA(cudaMemcpyAsync(c->stage + 2 * N, c->dMom, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    RT_BCUDA(cudaMemcpyAsync(&flags[i], c->flags, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  }
  RT_BCUDA(cudaStreamSynchronize(b->stream));
  const int keep = b->variant;
  double t[rtg::kBatchVariants];
  int best = -1;
  cudaEvent_t e0, e1;
  RT_BCUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return rtg::set_error(RT_E_CUDA, "rt_batch_autotune: event");
  }
  rt_status st = RT_OK;
  for (int v = 0; v < rtg::kBatchVariants && st == RT_OK; ++v) {
    t[v] = -1.0;
    b->variant = v;
    if (rebuild(b) != RT_OK) continue;   // this variant's tiles do not fit the largest angle set
    st = enqueue_step(b, 0);
    if (st == RT_OK && cudaEventRecord(e0, b->stream) != cudaSuccess) st = RT_E_CUDA;
    for (int k = 0; k < trial_steps && st == RT_OK; ++k) st = enqueue_step(b, 0);
    float el = 0;
    if (st == RT_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&el, e0, e1) != cudaSuccess))
      st = rtg::set_error(RT_E_CUDA, "rt_batch_autotune: timing");
    if (st != RT_OK) break;
    t[v] = (double)el / trial_steps;
    if (best < 0 || t[v] < t[best]) best = v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->variant = best >= 0 ? best : keep;
  b->dirty = true;
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    rt_ctx *c = b->ctxs[i];
    const size_t N = (size_t)c->N;
    RT_BCUDA(cudaMemcpyAsync(c->T, c->stage, N * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    RT_BCUDA(cudaMemcpyAsync(c->dEgas, c->stage + N, N * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    RT_BCUDA(cudaMemcpyAsync(c->dMom, c->stage + 2 * N, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    RT_BCUDA(cudaMemcpyAsync(c->flags, &flags[i], sizeof(int), cudaMemcpyHostToDevice, b->stream));
  }
  RT_BCUDA(cudaStreamSynchronize(b->stream));
  if (st != RT_OK) return st;
  if (best < 0) return rtg::set_error(RT_E_INVALID, "rt_batch_autotune: no variant fits the largest angle set");
  if (ms)
    for (int v = 0; v < rtg::kBatchVariants; ++v) ms[v] = t[v];
  if (chosen) *chosen = best;
  return RT_OK;
}

void rt_batch_destroy(rt_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (rt_ctx *c : b->ctxs) c->batch = nullptr;
  if (b->d_items) cudaFree(b->d_items);
  for (int p = 0; p < 2; ++p)
    if (b->d_desc[p]) cudaFree(b->d_desc[p]);
  delete b;
}

}  // extern "C"
