// Auto-tuning (Section 2.2: the tunable parameters are fixed by trying all
// meaningful combinations and keeping the fastest; Section 4.1: the optimum
// differs between platforms and observational setups).  dd_tune times every
// valid configuration of a plan with CUDA events (median of repeats, after a
// warm-up), most promising first, keeps the fastest, and can record / reuse
// the choice in a JSON-lines database keyed by device name and plan geometry.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dd_errors.h"
#include "dd_internal.h"

namespace dd {

static std::string tune_key(const dd_plan_s& p) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, p.device);
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s|C=%d|f_low=%.9g|chan_bw=%.9g|t_samp=%.9g|dm_first=%.9g|dm_step=%.9g|n_dm=%d|n_out=%lld|%s",
                prop.name, p.C, p.f_low, p.chan_bw, p.t_samp, p.dm_first, p.dm_step, p.n_dm, (long long)p.n_out,
                p.dtype == DD_U8_I32 ? "u8" : "f32");
  if (p.dm_index0 != 0)  // a plan over trials [dm_index0, dm_index0 + n_dm) of the grid
    std::snprintf(buf + std::strlen(buf), sizeof(buf) - std::strlen(buf), "|dm_index0=%d", p.dm_index0);
  return buf;
}

std::string tune_key_of(const dd_plan_s& p) { return tune_key(p); }

// Look for `"key": "<key>"` in the database; on a hit return the stored config name and time.
static bool db_lookup(const char* path, const std::string& key, std::string& cfg, double& ms) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  const std::string needle = "\"key\": \"" + key + "\"";
  std::vector<char> line(1 << 16);
  bool found = false;
  while (std::fgets(line.data(), (int)line.size(), f)) {
    const char* l = line.data();
    if (!std::strstr(l, needle.c_str())) continue;
    const char* c = std::strstr(l, "\"config\": \"");
    const char* t = std::strstr(l, "\"ms\": ");
    if (!c || !t) continue;
    c += std::strlen("\"config\": \"");
    const char* e = std::strchr(c, '"');
    if (!e) continue;
    cfg.assign(c, e);
    ms = std::atof(t + std::strlen("\"ms\": "));
    found = true;  // the last matching line wins
  }
  std::fclose(f);
  return found;
}

// A plan made while DD_TUNE_DB names a tuning database takes the choice
// recorded there for its device and geometry, if any (no timing is done).
void apply_tune_db(dd_plan_s* plan) {
  const char* path = std::getenv("DD_TUNE_DB");
  if (!path || !*path) return;
  std::string name;
  double ms = 0;
  if (!db_lookup(path, tune_key(*plan), name, ms)) return;
  for (size_t k = 0; k < plan->configs.size(); ++k)
    if (plan->configs[k].name == name) plan->selected = (int)k;
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_tune(dd_plan_t plan, double budget_s, const char* db_path, double* best_ms) {
  NvtxRange range("dd_tune");
  clear_error();
  if (!plan) return set_error(DD_ERR_ARG, "dd_tune: plan is NULL");
  const std::string key = tune_key(*plan);
  if (db_path) {
    std::string name;
    double ms = 0;
    if (db_lookup(db_path, key, name, ms)) {
      for (size_t k = 0; k < plan->configs.size(); ++k)
        if (plan->configs[k].name == name) {
          plan->selected = (int)k;
          if (best_ms) *best_ms = ms;
          return DD_OK;
        }
    }
  }
  const int elem = plan->dtype == DD_U8_I32 ? 1 : 4;
  // the stride every configuration takes as it is (no launch falls back to
  // another configuration, so each timing is the named configuration's)
  const int64_t stride = plan_in_stride(*plan);
  void* in = nullptr;
  void* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&in, (size_t)plan->C * stride * elem);
  if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)plan->n_dm * plan->n_out * 4);
  if (e == cudaSuccess) e = cudaMemset(in, 0x3c, (size_t)plan->C * stride * elem);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(in);
    cudaFree(out);
  };
  if (e != cudaSuccess) {
    cleanup();
    return set_error(DD_ERR_NOMEM, "dd_tune: cannot allocate timing buffers");
  }
  const auto wall0 = std::chrono::steady_clock::now();
  std::vector<double> med(plan->configs.size(), -1.0);
  int best = -1;
  // most promising configurations first, so that a time budget cut short
  // still has the good ones timed
  for (const int ki : config_preference_order(*plan)) {
    const size_t k = (size_t)ki;
    if (budget_s > 0 && best >= 0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - wall0).count();
      if (el > budget_s) break;
    }
    bool ok = true;
    for (int r = 0; r < 2 && ok; ++r)
      ok = forward_device(plan, in, stride, nullptr, out, plan->n_out, s, (int)k) == DD_OK;
    std::vector<float> t;
    for (int r = 0; r < 5 && ok; ++r) {
      cudaEventRecord(e0, s);
      ok = forward_device(plan, in, stride, nullptr, out, plan->n_out, s, (int)k) == DD_OK;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      t.push_back(ms);
    }
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    std::sort(t.begin(), t.end());
    med[k] = t[t.size() / 2];
    if (best < 0 || med[k] < med[best]) best = (int)k;
  }
  cleanup();
  clear_error();
  if (best < 0) return set_error(DD_ERR_CUDA, "dd_tune: no configuration ran");
  plan->selected = best;
  if (best_ms) *best_ms = med[best];
  if (db_path) {
    FILE* f = std::fopen(db_path, "a");
    if (f) {
      std::fprintf(f, "{\"key\": \"%s\", \"config\": \"%s\", \"ms\": %.6f, \"timings\": {", key.c_str(),
                   plan->configs[best].name.c_str(), med[best]);
      bool first = true;
      for (size_t k = 0; k < med.size(); ++k) {
        if (med[k] < 0) continue;
        std::fprintf(f, "%s\"%s\": %.6f", first ? "" : ", ", plan->configs[k].name.c_str(), med[k]);
        first = false;
      }
      std::fprintf(f, "}}\n");
      std::fclose(f);
    }
  }
  return DD_OK;
}
