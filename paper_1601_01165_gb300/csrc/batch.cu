// Batches: many independent beams (Section 2: every beam can be processed
// independently; Section 5.1: one device dedisperses many beams) launched as
// one CUDA graph.
//
// dd_batch_create orders the beams longest first (C * n_dm * n_out) and deals
// them to a few internal streams, each to the stream with the least work so
// far, so beams too small to fill the GPU run side by side.  dd_batch_run
// records, once per (pointer set, stream), the fork from the caller's stream,
// every beam's forward launch with its own plan's selected configuration on
// its internal stream, and the join back; later runs with the same pointers
// replay the graph with a single launch.  Each beam runs exactly the kernel
// dd_forward would run, so its output is bit-identical to dd_forward's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "dd_errors.h"
#include "dd_internal.h"

namespace {
constexpr int kBatchStreams = 4;
}

struct dd_batch_s {
  int device = 0;
  std::vector<dd_plan_t> plans;
  std::vector<int> order;            // beams, longest first
  std::vector<int> lane;             // internal stream of each beam
  cudaStream_t streams[kBatchStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kBatchStreams] = {};
  int n_streams = 0;
  // graph cache
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
  std::vector<const void*> key_in;
  std::vector<void*> key_out;
  std::vector<int64_t> key_in_stride, key_out_stride;
};

namespace dd {

static void free_batch(dd_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (int k = 0; k < b->n_streams; ++k) {
    if (b->streams[k]) cudaStreamDestroy(b->streams[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
}

// Fork from `s`, every beam's forward on its internal stream, join into `s`.
static dd_status launch_beams(dd_batch_s* b, const void* const* ins, const int64_t* in_strides, void* const* outs,
                              const int64_t* out_strides, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->fork, s);
  for (int k = 0; k < b->n_streams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: fork", e);
  for (int k : b->order) {
    const dd_status st = forward_device(b->plans[k], ins[k], in_strides[k], nullptr, outs[k], out_strides[k],
                                        b->streams[b->lane[k]], -1);
    if (st != DD_OK) return st;
  }
  for (int k = 0; k < b->n_streams && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->join[k], b->streams[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[k], 0);
  }
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: join", e);
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_batch_create(dd_batch_t* out, const dd_plan_t* plans, int32_t n) {
  clear_error();
  if (!out || !plans || n <= 0) return set_error(DD_ERR_ARG, "dd_batch_create: bad arguments");
  for (int32_t k = 0; k < n; ++k) {
    if (!plans[k]) return set_error(DD_ERR_ARG, "dd_batch_create: plan %d is NULL", k);
    if (plans[k]->device != plans[0]->device)
      return set_error(DD_ERR_ARG, "dd_batch_create: plans live on different devices");
  }
  dd_batch_s* b = new (std::nothrow) dd_batch_s();
  if (!b) return set_error(DD_ERR_NOMEM, "dd_batch_create: host allocation failed");
  b->plans.assign(plans, plans + n);
  b->device = plans[0]->device;
  // longest beams first, each to the least-loaded stream
  std::vector<double> cost(n);
  for (int32_t k = 0; k < n; ++k) cost[k] = (double)plans[k]->C * plans[k]->n_dm * (double)plans[k]->n_out;
  b->order.resize(n);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  b->n_streams = std::min<int>(kBatchStreams, n);
  b->lane.assign(n, 0);
  std::vector<double> load(b->n_streams, 0.0);
  for (int k : b->order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lane[k] = j;
    load[j] += cost[k];
  }
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess) e = cudaSetDevice(b->device);
  for (int k = 0; k < b->n_streams && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    free_batch(b);
    delete b;
    return set_cuda_error("dd_batch_create: streams", e);
  }
  *out = b;
  return DD_OK;
}

extern "C" dd_status dd_batch_run(dd_batch_t b, const void* const* ins, const int64_t* in_strides,
                                  void* const* outs, const int64_t* out_strides, void* stream) {
  NvtxRange range("dd_batch_run");
  clear_error();
  if (!b || !ins || !in_strides || !outs || !out_strides) return set_error(DD_ERR_ARG, "dd_batch_run: NULL argument");
  const size_t n = b->plans.size();
  for (size_t k = 0; k < n; ++k) {
    const dd_plan_s& p = *b->plans[k];
    const int elem = p.dtype == DD_U8_I32 ? 1 : 4;
    if (!ins[k] || !outs[k]) return set_error(DD_ERR_ARG, "dd_batch_run: beam %zu has a NULL buffer", k);
    if (in_strides[k] < p.n_in || out_strides[k] < p.n_out)
      return set_error(DD_ERR_SHAPE, "dd_batch_run: beam %zu strides too small", k);
    if ((uintptr_t)ins[k] % 16 != 0 || (in_strides[k] * elem) % 16 != 0)
      return set_error(DD_ERR_ALIGN, "dd_batch_run: beam %zu input must be 16-byte aligned with 16-byte row pitch", k);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool same = b->exec && b->exec_stream == s && b->key_in.size() == n &&
                    std::equal(b->key_in.begin(), b->key_in.end(), ins) &&
                    std::equal(b->key_out.begin(), b->key_out.end(), outs) &&
                    std::equal(b->key_in_stride.begin(), b->key_in_stride.end(), in_strides) &&
                    std::equal(b->key_out_stride.begin(), b->key_out_stride.end(), out_strides);
  cudaError_t e;
  if (same) {
    e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return set_cuda_error("dd_batch_run: graph launch", e);
    return DD_OK;
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->key_in.clear();
  if (s == nullptr) return launch_beams(b, ins, in_strides, outs, out_strides, s);  // the legacy stream: no capture
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: begin capture", e);
  const dd_status st = launch_beams(b, ins, in_strides, outs, out_strides, s);
  e = cudaStreamEndCapture(s, &graph);
  if (st != DD_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: end capture", e);
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return set_cuda_error("dd_batch_run: instantiate", e);
  }
  b->exec_stream = s;
  b->key_in.assign(ins, ins + n);
  b->key_out.assign(outs, outs + n);
  b->key_in_stride.assign(in_strides, in_strides + n);
  b->key_out_stride.assign(out_strides, out_strides + n);
  e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: graph launch", e);
  return DD_OK;
}

extern "C" dd_status dd_batch_tune(dd_batch_t b, double budget_s, const char* db_path, int32_t* n_tuned) {
  NvtxRange range("dd_batch_tune");
  clear_error();
  if (!b) return set_error(DD_ERR_ARG, "dd_batch_tune: batch is NULL");
  // one dd_tune per distinct setup (device, geometry, dtype), longest beams
  // first; every other beam of a setup takes the same configuration
  std::vector<std::pair<std::string, std::string>> done;  // key -> configuration name
  int32_t tuned = 0;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  dd_status st = DD_OK;
  for (int k : b->order) {
    dd_plan_s* p = b->plans[k];
    const std::string key = tune_key_of(*p);
    const std::string* name = nullptr;
    for (const auto& kv : done)
      if (kv.first == key) name = &kv.second;
    if (name) {
      for (size_t j = 0; j < p->configs.size(); ++j)
        if (p->configs[j].name == *name) p->selected = (int)j;
      continue;
    }
    st = dd_tune(p, budget_s, db_path, nullptr);
    if (st != DD_OK) break;
    done.emplace_back(key, p->configs[p->selected].name);
    ++tuned;
  }
  cudaSetDevice(prev);
  // the selections changed: record the graph again on the next run
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->key_in.clear();
  if (n_tuned) *n_tuned = tuned;
  return st;
}

extern "C" dd_status dd_batch_destroy(dd_batch_t b) {
  clear_error();
  if (!b) return DD_OK;
  free_batch(b);
  delete b;
  return DD_OK;
}
