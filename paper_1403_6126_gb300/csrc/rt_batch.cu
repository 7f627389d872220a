// Many independent problems advanced by one persistent launch per step.
//
// A batch holds contexts created with rt_create (float intensities).  For a
// step, a device work list names every (problem, tile) pair; a grid of
// persistent CTAs (one per SM at the shared-memory size the largest angle set
// needs) pulls items through an atomic counter and runs the same per-tile
// code as the single-problem kernel, so each problem's result is bitwise the
// one it gets alone.  Items are ordered by decreasing angle count so the long
// tiles start first.  Steps are captured in a CUDA graph (a counter reset and
// a kernel per step) and replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rt.h"
#include "rt_ctx.h"
#include "rt_step_pair.cuh"

namespace rtg {

struct WorkItem {
  int prob, tbx, tby, tbz;
};

// Tile shapes of the persistent kernel, per grid dimension.
constexpr int kB1X = 512;
constexpr int kB2X = 32, kB2Y = 16;
constexpr int kB3X = 16, kB3Y = 8, kB3Z = 4;
constexpr int kBatchThreads = 512;

template <bool VEL>
__global__ void __launch_bounds__(kBatchThreads, 1)
    batch_kernel(const StepArgs<float> *__restrict__ descs, const WorkItem *__restrict__ items, int nitems,
                 int *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ StepArgs<float> desc;
  __shared__ int s_item;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const WorkItem w = items[it];
    const int *src = reinterpret_cast<const int *>(descs + w.prob);
    int *dst = reinterpret_cast<int *>(&desc);
    for (int i = tid; i < (int)(sizeof(StepArgs<float>) / sizeof(int)); i += kBatchThreads) dst[i] = src[i];
    __syncthreads();
    if (desc.dim == 3)
      stepk::process_tile2<3, VEL, kB3X, kB3Y, kB3Z>(desc, tid, w.tbx, w.tby, w.tbz, smem);
    else if (desc.dim == 2)
      stepk::process_tile2<2, VEL, kB2X, kB2Y, 1>(desc, tid, w.tbx, w.tby, 0, smem);
    else
      stepk::process_tile2<1, VEL, kB1X, 1, 1>(desc, tid, w.tbx, 0, 0, smem);
    __syncthreads();   // every thread has read s_item and desc
  }
}

static_assert(kB1X == kBatchThreads && kB2X * kB2Y == kBatchThreads && kB3X * kB3Y * kB3Z == kBatchThreads,
              "every tile shape of the persistent kernel has one thread per cell");

bool batch_fits(int dim, int M, bool vel) {
  size_t sm = dim == 1   ? stepk::smem_bytes2(1, M, vel, kB1X, 1, 1)
              : dim == 2 ? stepk::smem_bytes2(2, M, vel, kB2X, kB2Y, 1)
                         : stepk::smem_bytes2(3, M, vel, kB3X, kB3Y, kB3Z);
  return sm <= 227 * 1024;
}

}  // namespace rtg

struct rt_batch {
  cudaStream_t stream = nullptr;
  std::vector<rt_ctx *> ctxs;
  bool dirty = true;
  bool vel = false;
  int nitems = 0, grid = 0, phase = 0;
  size_t smem = 0;
  rtg::WorkItem *d_items = nullptr;
  rtg::StepArgs<float> *d_desc[2] = {nullptr, nullptr};
  int *d_counter = nullptr;
  size_t items_cap = 0, desc_cap = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0, graph_phase = -1;
};

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
  drop_graph(b);
  std::vector<int> order(b->ctxs.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->ctxs[x]->M > b->ctxs[y]->M; });
  std::vector<rtg::WorkItem> items;
  int Mmax = 1;
  bool dims[4] = {false, false, false, false};
  b->vel = false;
  for (rt_ctx *c : b->ctxs) b->vel = b->vel || rtg::velocity_on(c);
  for (int i : order) {
    rt_ctx *c = b->ctxs[i];
    Mmax = std::max(Mmax, c->M);
    dims[c->dim] = true;
    int tx = c->dim == 1 ? rtg::kB1X : c->dim == 2 ? rtg::kB2X : rtg::kB3X;
    int ty = c->dim == 2 ? rtg::kB2Y : c->dim == 3 ? rtg::kB3Y : 1;
    int tz = c->dim == 3 ? rtg::kB3Z : 1;
    for (int z = 0; z < (c->n[2] + tz - 1) / tz; ++z)
      for (int y = 0; y < (c->n[1] + ty - 1) / ty; ++y)
        for (int x = 0; x < (c->n[0] + tx - 1) / tx; ++x) items.push_back({i, x, y, z});
  }
  size_t smem = 0;
  if (dims[1]) smem = std::max(smem, rtg::stepk::smem_bytes2(1, Mmax, b->vel, rtg::kB1X, 1, 1));
  if (dims[2]) smem = std::max(smem, rtg::stepk::smem_bytes2(2, Mmax, b->vel, rtg::kB2X, rtg::kB2Y, 1));
  if (dims[3]) smem = std::max(smem, rtg::stepk::smem_bytes2(3, Mmax, b->vel, rtg::kB3X, rtg::kB3Y, rtg::kB3Z));
  if (smem > 227 * 1024)
    return rtg::set_error(RT_E_INVALID, "rt_batch: the largest angle set does not fit the batch tile in shared memory");
  b->smem = smem;
  b->nitems = (int)items.size();
  if (items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    RT_BCUDA(cudaMalloc(&b->d_items, sizeof(rtg::WorkItem) * items.size()));
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
    for (int p = 0; p < 2; ++p) {
      if (b->d_desc[p]) cudaFree(b->d_desc[p]);
      b->d_desc[p] = nullptr;
      RT_BCUDA(cudaMalloc(&b->d_desc[p], sizeof(rtg::StepArgs<float>) * b->ctxs.size()));
    }
    b->desc_cap = b->ctxs.size();
  }
  for (int p = 0; p < 2; ++p)
    if (!desc[p].empty())
      RT_BCUDA(cudaMemcpyAsync(b->d_desc[p], desc[p].data(), sizeof(rtg::StepArgs<float>) * desc[p].size(),
                               cudaMemcpyHostToDevice, b->stream));
  RT_BCUDA(cudaStreamSynchronize(b->stream));
  auto kern = b->vel ? rtg::batch_kernel<true> : rtg::batch_kernel<false>;
  RT_BCUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int per_sm = 0, dev = 0, sms = 0;
  RT_BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, rtg::kBatchThreads, b->smem));
  RT_BCUDA(cudaGetDevice(&dev));
  RT_BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  b->grid = std::max(1, std::min(b->nitems, sms * std::max(1, per_sm)));
  b->phase = 0;
  b->dirty = false;
  return RT_OK;
}

// Queues one step: counter reset and one persistent launch.
rt_status enqueue_step(rt_batch *b, int parity) {
  RT_BCUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream));
  auto kern = b->vel ? rtg::batch_kernel<true> : rtg::batch_kernel<false>;
  kern<<<b->grid, rtg::kBatchThreads, b->smem, b->stream>>>(b->d_desc[parity], b->d_items, b->nitems, b->d_counter);
  RT_BCUDA(cudaGetLastError());
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
  if (cudaMalloc(&b->d_counter, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return rtg::set_error(RT_E_NOMEM, "rt_batch_create: device allocation");
  }
  *out = b;
  return RT_OK;
}

rt_status rt_batch_add(rt_batch *b, rt_ctx *c) {
  if (!b || !c) return rtg::set_error(RT_E_INVALID, "rt_batch_add: NULL argument");
  if (c->fp64) return rtg::set_error(RT_E_INVALID, "rt_batch_add: batches run float intensities (RT_FP32)");
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

void rt_batch_destroy(rt_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (rt_ctx *c : b->ctxs) c->batch = nullptr;
  if (b->d_items) cudaFree(b->d_items);
  for (int p = 0; p < 2; ++p)
    if (b->d_desc[p]) cudaFree(b->d_desc[p]);
  if (b->d_counter) cudaFree(b->d_counter);
  delete b;
}

}  // extern "C"
