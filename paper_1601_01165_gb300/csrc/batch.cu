// Batches: many independent beams (Section 2: every beam can be processed
// independently; Section 5.1: one device dedisperses many beams) launched as
// one CUDA graph.
//
// dd_batch_create orders the beams longest first (C * n_dm * n_out).  Each
// beam runs the configuration dd_forward would run for it (its plan's
// selection, e.g. from dd_batch_tune, resolved for its input layout), so its
// output is bit-identical to dd_forward's.  Beams whose configurations have a
// persistent form (the staged, packed-uint8 and 9-trial Tensor-Memory
// kernels) can share one persistent launch per configuration group: its
// blocks take the group's tiles, longest beam first, from a work counter
// until none are left, so small beams fill the tails of large ones.  A group
// runs that way where dd_batch_tune measured it faster than its beams' own
// launches (or wherever it can, in mode 2); other beams get one launch each.  The launches are dealt to a few internal streams by
// accumulated work.  dd_batch_run records, once per (pointer set, stream),
// the fork from the caller's stream, the counter resets and launches, and the
// join back; later runs with the same pointers replay the graph with a single
// launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <functional>
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
  int sms = 0;
  int mode = 1;                      // persistent launches: 0 never, 1 auto, 2 wherever a group can have one
  std::vector<std::pair<std::string, bool>> choice;  // auto mode: group key -> persistent (measured by dd_batch_tune)
  std::vector<dd_plan_t> plans;
  std::vector<int> order;            // beams, longest first
  std::vector<double> cost;          // C * n_dm * n_out of each beam
  void* dev = nullptr;               // persistent work: tensor maps, counters
  size_t dev_bytes = 0;
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
  cudaFree(b->dev);
  for (int k = 0; k < b->n_streams; ++k) {
    if (b->streams[k]) cudaStreamDestroy(b->streams[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
}

// One persistent launch: up to kBeamsPerLaunch beams of one configuration and dtype.
struct Group {
  const TileConfig* cfg = nullptr;
  dd_dtype dtype = DD_F32_F32;
  std::vector<BatchBeam> beams;  // longest first
  std::vector<int> ks;           // their beam numbers in the batch
  std::string key;               // configuration, dtype and blocks per SM
  int n_items = 0;
  int smem = 0;
  int per_sm = 0;  // resident blocks per SM of every member at its own shared memory
  int grid = 0;
  double cost = 0;
  size_t off_maps = 0, off_counter = 0;
};

// The launches of one run: persistent groups and single beams, with their
// device work uploaded.  Called outside any stream capture.
struct RunPlan {
  std::vector<Group> groups;
  std::vector<int> singles;  // beams launched one by one
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Does a group run as one persistent launch?  Mode 2: yes; mode 1: if
// dd_batch_tune measured it faster than its beams' own launches (untimed
// groups run one launch per beam: on GB300 no kind's persistent launch
// measured reliably faster).
static bool group_persistent(const dd_batch_s* b, const std::string& key) {
  if (b->mode == 2) return true;
  for (const auto& kv : b->choice)
    if (kv.first == key) return kv.second;
  return false;
}

// Sort the beams into persistent groups and single launches for the given
// buffers, and upload the groups' tensor maps and counters (synchronizing
// `s` first: an earlier run may still read them).
static dd_status build_run(dd_batch_s* b, const void* const* ins, const int64_t* in_strides, void* const* outs,
                           const int64_t* out_strides, cudaStream_t s, RunPlan& rp) {
  rp.groups.clear();
  rp.singles.clear();
  std::vector<std::vector<char>> maps;  // per group, host copies of TMW9 tensor maps
  for (int k : b->order) {
    dd_plan_s* p = b->plans[k];
    const FwdArgs a = plan_args(p, ins[k], in_strides[k], nullptr, outs[k], out_strides[k], 0, p->n_out);
    const TileConfig* cfg = resolve_config(p, a, -1);
    if (b->mode == 0 || !has_persistent(*cfg, p->dtype)) {
      rp.singles.push_back(k);
      continue;
    }
    // A beam joins a persistent launch only if the persistent kernel keeps
    // its plain launch's blocks per SM; beams of one configuration share a
    // launch when their own shared memory gives the same blocks per SM (the
    // launch takes its largest member's shared memory, so none loses any).
    const int smem = persistent_smem(*cfg, p->dtype, cfg->pitch);
    const int per_sm = persistent_blocks_per_sm(*cfg, p->dtype, smem);
    const std::string key = cfg->name + (p->dtype == DD_U8_I32 ? "/u8/" : "/f32/") + std::to_string(per_sm);
    if (per_sm < 1 || per_sm < plain_blocks_per_sm(*cfg, p->dtype, cfg->smem) || !group_persistent(b, key)) {
      rp.singles.push_back(k);
      continue;
    }
    size_t gi = 0;
    while (gi < rp.groups.size() &&
           !(rp.groups[gi].key == key && rp.groups[gi].beams.size() < (size_t)kBeamsPerLaunch))
      ++gi;
    if (gi == rp.groups.size()) {
      rp.groups.emplace_back();
      rp.groups.back().cfg = cfg;
      rp.groups.back().dtype = p->dtype;
      rp.groups.back().per_sm = per_sm;
      rp.groups.back().key = key;
      maps.emplace_back();
    }
    Group& g = rp.groups[gi];
    BatchBeam bm{};
    bm.a = a;
    bm.pitch = cfg->pitch;
    // the plain launch's grid: (time tiles, DM blocks), or (9-trial groups, time tiles) for TMW9
    const int64_t nt = (p->n_out + cfg->bt - 1) / cfg->bt, nd = (p->n_dm + cfg->bd - 1) / cfg->bd;
    const bool dm_x = cfg->kind == Kind::TmW9;
    bm.nx = (int)(dm_x ? nd : nt);
    bm.first = g.n_items;
    const int64_t items = nt * nd;
    if (g.n_items + items > (int64_t)1 << 30) return set_error(DD_ERR_SHAPE, "dd_batch_run: too many tiles");
    if (cfg->kind == Kind::TmW9) {
      std::vector<char>& mv = maps[gi];
      const size_t at = mv.size();
      mv.resize(at + tmw9_views_bytes());
      if (!tmw9_encode_views(a, mv.data() + at))
        return set_error(DD_ERR_CUDA, "dd_batch_run: beam %d: cannot encode its tensor maps", k);
    }
    g.n_items += (int)items;
    g.smem = std::max(g.smem, smem);
    g.cost += b->cost[k];
    g.beams.push_back(bm);
    g.ks.push_back(k);
  }
  for (Group& g : rp.groups) g.grid = (int)std::min<int64_t>(g.n_items, (int64_t)g.per_sm * b->sms);
  // device layout: per group its tensor maps (64-byte aligned), then one
  // counter per group (the beams travel in the launch's parameters)
  size_t bytes = 0;
  for (size_t gi = 0; gi < rp.groups.size(); ++gi) {
    Group& g = rp.groups[gi];
    g.off_maps = bytes = align_up(bytes, 64);
    bytes += maps[gi].size();
  }
  for (Group& g : rp.groups) {
    g.off_counter = bytes = align_up(bytes, 16);
    bytes += sizeof(int);
  }
  if (rp.groups.empty()) return DD_OK;
  std::vector<char> host(bytes, 0);
  for (size_t gi = 0; gi < rp.groups.size(); ++gi) {
    Group& g = rp.groups[gi];
    if (!maps[gi].empty()) std::memcpy(host.data() + g.off_maps, maps[gi].data(), maps[gi].size());
  }
  // earlier runs may still read the old work: let them finish before it changes
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && b->dev_bytes < bytes) {
    cudaFree(b->dev);
    b->dev = nullptr;
    b->dev_bytes = 0;
    e = cudaMalloc(&b->dev, bytes);
    if (e == cudaSuccess) b->dev_bytes = bytes;
  }
  if (e == cudaSuccess) e = cudaMemcpy(b->dev, host.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: work upload", e);
  return DD_OK;
}

// Fork from `s`, the run's launches on the internal streams (persistent
// groups and single beams dealt by accumulated work), join into `s`.
static dd_status launch_run(dd_batch_s* b, const RunPlan& rp, const void* const* ins, const int64_t* in_strides,
                            void* const* outs, const int64_t* out_strides, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->fork, s);
  for (int k = 0; k < b->n_streams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: fork", e);
  std::vector<double> load(b->n_streams, 0.0);
  auto pick = [&](double cost) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[j] += cost;
    return b->streams[j];
  };
  char* dev = static_cast<char*>(b->dev);
  for (const Group& g : rp.groups) {
    cudaStream_t st = pick(g.cost);
    BatchWork w{};
    w.maps = g.cfg->kind == Kind::TmW9 ? static_cast<const void*>(dev + g.off_maps) : nullptr;
    w.n_beams = (int)g.beams.size();
    std::copy(g.beams.begin(), g.beams.end(), w.beams);
    w.n_items = g.n_items;
    w.counter = reinterpret_cast<int*>(dev + g.off_counter);
    e = cudaMemsetAsync(w.counter, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_persistent(*g.cfg, g.dtype, w, g.smem, g.grid, st);
    if (e != cudaSuccess) return set_cuda_error("dd_batch_run: persistent launch", e);
  }
  for (int k : rp.singles) {
    const dd_status st = forward_device(b->plans[k], ins[k], in_strides[k], nullptr, outs[k], out_strides[k],
                                        pick(b->cost[k]), -1);
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
  // longest beams first (each run deals its launches to the least-loaded stream)
  std::vector<double>& cost = b->cost;
  cost.resize(n);
  for (int32_t k = 0; k < n; ++k) cost[k] = (double)plans[k]->C * plans[k]->n_dm * (double)plans[k]->n_out;
  b->order.resize(n);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  b->n_streams = std::min<int>(kBatchStreams, n);
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess) e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
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
  RunPlan rp;
  dd_status st = build_run(b, ins, in_strides, outs, out_strides, s, rp);
  if (st != DD_OK) return st;
  if (s == nullptr) return launch_run(b, rp, ins, in_strides, outs, out_strides, s);  // the legacy stream: no capture
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return set_cuda_error("dd_batch_run: begin capture", e);
  st = launch_run(b, rp, ins, in_strides, outs, out_strides, s);
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

// Time each persistent group of the batch's current selections against its
// beams' own launches, one after another on one stream (best of three each,
// on scratch buffers sized for the largest beam), and keep the persistent
// launch where it was faster.  Without the scratch memory nothing is timed
// and the kinds' defaults stay.
static dd_status tune_persistent(dd_batch_s* b) {
  b->choice.clear();
  const size_t n = b->plans.size();
  size_t in_bytes = 16, out_bytes = 16;
  std::vector<int64_t> in_strides(n), out_strides(n);
  for (size_t k = 0; k < n; ++k) {
    const dd_plan_s& p = *b->plans[k];
    in_strides[k] = plan_in_stride(p);
    out_strides[k] = p.n_out;
    in_bytes = std::max(in_bytes, (size_t)p.C * (size_t)in_strides[k] * (p.dtype == DD_U8_I32 ? 1 : 4));
    out_bytes = std::max(out_bytes, (size_t)p.n_dm * (size_t)p.n_out * 4);
  }
  void *in = nullptr, *out = nullptr;
  if (cudaMalloc(&in, in_bytes) != cudaSuccess || cudaMalloc(&out, out_bytes) != cudaSuccess) {
    cudaFree(in);
    cudaGetLastError();  // not an error of the call: the defaults stay
    return DD_OK;
  }
  cudaStream_t s = b->streams[0];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(in, 0, in_bytes, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<const void*> ins(n, in);
  std::vector<void*> outs(n, out);
  const int mode = b->mode;
  b->mode = 2;  // every group that can be persistent
  RunPlan rp;
  dd_status st = e == cudaSuccess ? DD_OK : set_cuda_error("dd_batch_tune: scratch", e);
  if (st == DD_OK) st = cudaDeviceSynchronize() == cudaSuccess ? DD_OK : set_error(DD_ERR_CUDA, "dd_batch_tune: sync");
  if (st == DD_OK) st = build_run(b, ins.data(), in_strides.data(), outs.data(), out_strides.data(), s, rp);
  b->mode = mode;
  char* dev = static_cast<char*>(b->dev);
  auto best_of_3 = [&](const std::function<dd_status()>& run, float& ms) -> dd_status {
    ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return set_error(DD_ERR_CUDA, "dd_batch_tune: event");
      const dd_status r = run();
      if (r != DD_OK) return r;
      float t = 0;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        return set_error(DD_ERR_CUDA, "dd_batch_tune: timing");
      ms = std::min(ms, t);
    }
    return DD_OK;
  };
  for (size_t gi = 0; gi < rp.groups.size() && st == DD_OK; ++gi) {
    const Group& g = rp.groups[gi];
    float t_persist = 0, t_plain = 0;
    st = best_of_3(
        [&]() {
          BatchWork w{};
          w.maps = g.cfg->kind == Kind::TmW9 ? static_cast<const void*>(dev + g.off_maps) : nullptr;
          w.n_beams = (int)g.beams.size();
          w.n_items = g.n_items;
          w.counter = reinterpret_cast<int*>(dev + g.off_counter);
          std::copy(g.beams.begin(), g.beams.end(), w.beams);
          cudaError_t r = cudaMemsetAsync(w.counter, 0, sizeof(int), s);
          if (r == cudaSuccess) r = launch_persistent(*g.cfg, g.dtype, w, g.smem, g.grid, s);
          return r == cudaSuccess ? DD_OK : set_cuda_error("dd_batch_tune: persistent launch", r);
        },
        t_persist);
    if (st == DD_OK)
      st = best_of_3(
          [&]() {
            for (int k : g.ks) {
              const dd_status r = forward_device(b->plans[k], in, in_strides[k], nullptr, out, out_strides[k], s, -1);
              if (r != DD_OK) return r;
            }
            return DD_OK;
          },
          t_plain);
    if (st == DD_OK) b->choice.emplace_back(g.key, t_persist < t_plain);
  }
  cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(in);
  cudaFree(out);
  return st;
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
  if (st == DD_OK) st = tune_persistent(b);
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

extern "C" dd_status dd_batch_set_persistent(dd_batch_t b, int32_t mode) {
  clear_error();
  if (!b) return set_error(DD_ERR_ARG, "dd_batch_set_persistent: batch is NULL");
  if (mode < 0 || mode > 2) return set_error(DD_ERR_ARG, "dd_batch_set_persistent: mode must be 0, 1 or 2");
  b->mode = mode;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->key_in.clear();
  return DD_OK;
}

extern "C" dd_status dd_batch_destroy(dd_batch_t b) {
  clear_error();
  if (!b) return DD_OK;
  free_batch(b);
  delete b;
  return DD_OK;
}
