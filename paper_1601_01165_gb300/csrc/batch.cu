// Batches: many independent beams (Section 2: every beam can be processed
// independently; Section 5.1: one device dedisperses many beams) in one
// persistent launch per input type, captured in a CUDA graph.
//
// dd_batch_create sorts the beams into groups by input type and by how many
// blocks per SM their shared-memory need allows, and turns each group into a
// work list of (beam, DM block, time block) tiles, longest beam first (big
// beams start early, small ones fill the tail) with a persistent grid sized
// by that occupancy.  dd_batch_run writes the beams' pointers into a device
// descriptor table and launches; the launch sequence (counter reset +
// persistent kernels) is captured once per (pointer set, stream) and replayed
// afterwards.  Every tile is computed exactly as the solo kernels do, so a
// beam's output is bit-identical to dd_forward on its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "dd_errors.h"
#include "dd_internal.h"

namespace dd {
int32_t block_spread_of(const dd_plan_s& p, int bd);
}

struct dd_batch_s {
  int device = 0;
  std::vector<dd_plan_t> plans;
  struct Group {
    dd_dtype dtype;
    dd::TileConfig cfg;
    std::vector<int> beams;      // indices into plans
    std::vector<int> pitch;      // per beam in the group
    int smem = 0;
    int grid = 0;
    int n_items = 0;
    dd::BatchItem* d_items = nullptr;
    dd::BatchBeam* d_beams = nullptr;
    dd::BatchBeam* h_beams = nullptr;  // page-locked staging
  };
  std::vector<Group> groups;
  int* d_counters = nullptr;  // one per group
  int* d_status = nullptr;    // the first plan's device status word (not owned)
  // graph cache
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
  std::vector<const void*> key_in;
  std::vector<void*> key_out;
  std::vector<int64_t> key_in_stride, key_out_stride;
};

namespace dd {

static void free_batch(dd_batch_s* b) {
  for (auto& g : b->groups) {
    cudaFree(g.d_items);
    cudaFree(g.d_beams);
    cudaFreeHost(g.h_beams);
  }
  cudaFree(b->d_counters);
  if (b->exec) cudaGraphExecDestroy(b->exec);
}

static dd_status launch_groups(dd_batch_s* b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_counters, 0, b->groups.size() * sizeof(int), s);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: counter reset", e);
  for (size_t k = 0; k < b->groups.size(); ++k) {
    auto& g = b->groups[k];
    e = launch_batch(g.dtype, g.d_beams, g.d_items, g.n_items, b->d_counters + k, b->d_status, g.smem, g.grid, s);
    if (e != cudaSuccess) return set_cuda_error("dd_batch_run: launch", e);
  }
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_batch_create(dd_batch_t* out, const dd_plan_t* plans, int32_t n) {
  clear_error();
  if (!out || !plans || n <= 0) return set_error(DD_ERR_ARG, "dd_batch_create: bad arguments");
  dd_batch_s* b = new (std::nothrow) dd_batch_s();
  if (!b) return set_error(DD_ERR_NOMEM, "dd_batch_create: host allocation failed");
  b->plans.assign(plans, plans + n);
  for (int32_t k = 0; k < n; ++k) {
    if (!plans[k]) {
      delete b;
      return set_error(DD_ERR_ARG, "dd_batch_create: plan %d is NULL", k);
    }
    if (plans[k]->device != plans[0]->device) {
      delete b;
      return set_error(DD_ERR_ARG, "dd_batch_create: plans live on different devices");
    }
  }
  b->device = plans[0]->device;
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    delete b;
    return set_cuda_error("dd_batch_create: device query", e);
  }
  // One group per (input type, occupancy class): beams whose shared-memory
  // need allows the same number of resident blocks per SM share a persistent
  // launch, so a wide-spread beam does not lower the occupancy of the others.
  for (dd_dtype dt : {DD_F32_F32, DD_U8_I32}) {
    const TileConfig cfg = batch_config(dt);
    const int V = dt == DD_U8_I32 ? 16 : 4;
    const int slack = dt == DD_U8_I32 ? 32 : 0;
    struct BeamInfo {
      int k, pitch, smem, per_sm;
      double cost;
    };
    std::vector<BeamInfo> infos;
    for (int32_t k = 0; k < n; ++k) {
      const dd_plan_s& p = *plans[k];
      if (p.dtype != dt) continue;
      const int64_t spread = block_spread_of(p, cfg.bd);
      const int64_t pitch = (cfg.bt + spread + 2 * V + slack + V - 1) / V * V;
      const int smem = batch_smem_for(dt, (int)pitch);
      if (smem > kMaxSmemPerBlock) {
        free_batch(b);
        delete b;
        return set_error(DD_ERR_UNSUPPORTED, "dd_batch_create: beam %d needs %d bytes of shared memory", k, smem);
      }
      infos.push_back({k, (int)pitch, smem, std::max(1, batch_blocks_per_sm(dt, smem)),
                       (double)p.C * p.n_dm * p.n_out});
    }
    std::vector<int> classes;
    for (const auto& bi : infos)
      if (std::find(classes.begin(), classes.end(), bi.per_sm) == classes.end()) classes.push_back(bi.per_sm);
    std::sort(classes.begin(), classes.end());
    for (int per_sm : classes) {
      dd_batch_s::Group g;
      g.dtype = dt;
      g.cfg = cfg;
      std::vector<BeamInfo> mine;
      for (const auto& bi : infos)
        if (bi.per_sm == per_sm) mine.push_back(bi);
      // longest beams first (largest C * n_dm * n_out)
      std::stable_sort(mine.begin(), mine.end(), [](const BeamInfo& x, const BeamInfo& y) { return x.cost > y.cost; });
      std::vector<BatchItem> items;
      for (size_t j = 0; j < mine.size(); ++j) {
        const dd_plan_s& p = *plans[mine[j].k];
        g.beams.push_back(mine[j].k);
        g.pitch.push_back(mine[j].pitch);
        g.smem = std::max(g.smem, mine[j].smem);
        const int32_t td = (p.n_dm + cfg.bd - 1) / cfg.bd;
        const int64_t tt = (p.n_out + cfg.bt - 1) / cfg.bt;
        for (int32_t d = 0; d < td; ++d)
          for (int64_t t = 0; t < tt; ++t) items.push_back(BatchItem{(int32_t)j, d, (int32_t)t, 0});
      }
      if (items.size() > (size_t)INT32_MAX) {
        free_batch(b);
        delete b;
        return set_error(DD_ERR_UNSUPPORTED, "dd_batch_create: too many tiles");
      }
      g.n_items = (int)items.size();
      g.grid = std::max(1, std::min(sms * per_sm, g.n_items));
      e = cudaMalloc(&g.d_items, items.size() * sizeof(BatchItem));
      if (e == cudaSuccess)
        e = cudaMemcpy(g.d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMalloc(&g.d_beams, g.beams.size() * sizeof(BatchBeam));
      if (e == cudaSuccess) e = cudaMallocHost(&g.h_beams, g.beams.size() * sizeof(BatchBeam));
      b->groups.push_back(g);
      if (e != cudaSuccess) {
        free_batch(b);
        delete b;
        return set_error(DD_ERR_NOMEM, "dd_batch_create: allocation failed");
      }
    }
  }
  b->d_status = plans[0]->d_status;
  e = cudaMalloc(&b->d_counters, b->groups.size() * sizeof(int));
  if (e != cudaSuccess) {
    free_batch(b);
    delete b;
    return set_error(DD_ERR_NOMEM, "dd_batch_create: allocation failed");
  }
  *out = b;
  return DD_OK;
}

extern "C" dd_status dd_batch_run(dd_batch_t b, const void* const* ins, const int64_t* in_strides,
                                  void* const* outs, const int64_t* out_strides, void* stream) {
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
  // new pointer set: refresh the device descriptors (ordered on the stream
  // after any earlier run on it), then capture and launch
  for (auto& g : b->groups) {
    for (size_t j = 0; j < g.beams.size(); ++j) {
      const int k = g.beams[j];
      const dd_plan_s& p = *b->plans[k];
      BatchBeam bb{};
      bb.in = ins[k];
      bb.in_stride = in_strides[k];
      bb.out = outs[k];
      bb.out_stride = out_strides[k];
      bb.delaysT = p.d_delaysT;
      bb.C = p.C;
      bb.n_dm = p.n_dm;
      bb.n_dm_pad = p.n_dm_pad;
      bb.pitch = g.pitch[j];
      bb.n_out = p.n_out;
      bb.n_in = p.n_in;
      g.h_beams[j] = bb;
    }
    e = cudaMemcpyAsync(g.d_beams, g.h_beams, g.beams.size() * sizeof(BatchBeam), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return set_cuda_error("dd_batch_run: descriptor upload", e);
  }
  // the page-locked descriptors must not change while the copy is pending
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: synchronize", e);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->key_in.assign(ins, ins + n);
  b->key_out.assign(outs, outs + n);
  b->key_in_stride.assign(in_strides, in_strides + n);
  b->key_out_stride.assign(out_strides, out_strides + n);
  if (s == nullptr) {  // the legacy stream cannot be captured: launch directly
    b->key_in.clear();
    return launch_groups(b, s);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: begin capture", e);
  dd_status st = launch_groups(b, s);
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
  e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: graph launch", e);
  return DD_OK;
}

extern "C" dd_status dd_batch_destroy(dd_batch_t b) {
  clear_error();
  if (!b) return DD_OK;
  free_batch(b);
  delete b;
  return DD_OK;
}
