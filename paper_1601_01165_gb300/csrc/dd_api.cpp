// C ABI: errors, forward on device buffers and on host buffers.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "dd_errors.h"
#include "dd_internal.h"

namespace dd {

static thread_local std::string g_last_error;

dd_status set_error(dd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

dd_status set_cuda_error(const char* where, cudaError_t e) {
  if (e == cudaSuccess) e = cudaGetLastError();
  return set_error(DD_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_last_error.clear(); }

FwdArgs plan_args(const dd_plan_s* p, const void* in, int64_t in_stride, const float* w, void* out,
                  int64_t out_stride, int64_t t0, int64_t t1) {
  const int elem = p->dtype == DD_U8_I32 ? 1 : 4;
  FwdArgs a{};
  a.in = static_cast<const unsigned char*>(in) + t0 * elem;
  a.in_stride = in_stride;
  a.in_avail = in_stride - t0;
  a.w = w;
  a.out = static_cast<unsigned char*>(out) + t0 * 4;
  a.out_stride = out_stride;
  a.delays = p->d_delays;
  a.delaysT = p->d_delaysT;
  a.hex_desc = p->d_hex_desc;
  a.nine_desc = p->d_nine_desc;
  a.C = p->C;
  a.n_dm = p->n_dm;
  a.n_dm_pad = p->n_dm_pad;
  a.n_out = t1 - t0;
  a.n_in = (t1 - t0) + p->max_delay;
  a.status = p->d_status;
  return a;
}

const TileConfig* resolve_config(const dd_plan_s* p, const FwdArgs& a, int cfg_override) {
  const int elem = p->dtype == DD_U8_I32 ? 1 : 4;
  const int k = cfg_override >= 0 ? cfg_override : p->selected;
  const TileConfig* cfg = &p->configs[k];
  // Bulk copies need a 16-byte aligned source and row pitch; otherwise use the
  // plain-load kernel, which computes the same sums.
  const bool aligned = ((uintptr_t)a.in % 16 == 0) && ((a.in_stride * elem) % 16 == 0);
  auto first_of = [&](Kind kind) -> const TileConfig* {
    for (size_t j = 0; j < p->configs.size(); ++j)
      if (p->configs[j].kind == kind) return &p->configs[j];
    return nullptr;
  };
  if (cfg->kind != Kind::Naive && !aligned) cfg = first_of(Kind::Naive);
  // TMW9 needs spare samples after each row, else TMW6 (if offered) takes it;
  // TMW6 stages 128-byte rows; other layouts take the preferred shared-memory kernel
  if (cfg->kind == Kind::TmW9 && !tmw9_accepts(a.in, a.in_stride, a.n_in)) {
    const TileConfig* t6 = first_of(Kind::TmW6);
    cfg = t6 ? t6 : &p->configs[p->fallback];
  }
  if (cfg->kind == Kind::TmW6 && !tmw6_accepts(a.in, a.in_stride)) cfg = &p->configs[p->fallback];
  return cfg;
}

// Launch of the selected (or a fallback) forward kernel over output samples
// [t0, t1) (arguments already validated; t0 a multiple of 4096 samples keeps
// every alignment the kernels rely on).
static dd_status launch_range(dd_plan_s* p, const void* in, int64_t in_stride, const float* w, void* out,
                              int64_t out_stride, int64_t t0, int64_t t1, cudaStream_t stream, int cfg_override) {
  const FwdArgs a = plan_args(p, in, in_stride, w, out, out_stride, t0, t1);
  const TileConfig* cfg = resolve_config(p, a, cfg_override);
  cudaError_t e = launch_forward(*cfg, p->dtype, a, stream);
  if (e != cudaSuccess) return set_cuda_error("dd_forward: launch", e);
  return DD_OK;
}

// Validated launch of the selected (or a fallback) forward kernel.
dd_status forward_device(dd_plan_s* p, const void* in, int64_t in_stride, const float* w, void* out,
                         int64_t out_stride, cudaStream_t stream, int cfg_override) {
  if (!in || !out) return set_error(DD_ERR_ARG, "dd_forward: in/out is NULL");
  if (in_stride < p->n_in)
    return set_error(DD_ERR_SHAPE, "dd_forward: in_row_stride %lld < n_in %lld", (long long)in_stride,
                     (long long)p->n_in);
  if (out_stride < p->n_out)
    return set_error(DD_ERR_SHAPE, "dd_forward: out_row_stride %lld < n_out %lld", (long long)out_stride,
                     (long long)p->n_out);
  if (p->dtype == DD_U8_I32 && w)
    return set_error(DD_ERR_UNSUPPORTED, "dd_forward: uint8 plans take unit weights only (w must be NULL)");
  return launch_range(p, in, in_stride, w, out, out_stride, 0, p->n_out, stream, cfg_override);
}

}  // namespace dd

using namespace dd;

extern "C" const char* dd_status_string(dd_status s) {
  switch (s) {
    case DD_OK: return "DD_OK";
    case DD_ERR_ARG: return "DD_ERR_ARG";
    case DD_ERR_SHAPE: return "DD_ERR_SHAPE";
    case DD_ERR_ALIGN: return "DD_ERR_ALIGN";
    case DD_ERR_NOMEM: return "DD_ERR_NOMEM";
    case DD_ERR_CUDA: return "DD_ERR_CUDA";
    case DD_ERR_UNSUPPORTED: return "DD_ERR_UNSUPPORTED";
    case DD_ERR_BUDGET: return "DD_ERR_BUDGET";
    case DD_ERR_STATE: return "DD_ERR_STATE";
  }
  return "DD_ERR_UNKNOWN";
}

extern "C" const char* dd_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* dd_version(void) { return "libdd 0.1 (sm_103a)"; }

extern "C" dd_status dd_forward(dd_plan_t plan, const void* in, int64_t in_row_stride, const float* w, void* out,
                                int64_t out_row_stride, void* stream) {
  NvtxRange range("dd_forward");
  clear_error();
  if (!plan) return set_error(DD_ERR_ARG, "dd_forward: plan is NULL");
  return forward_device(plan, in, in_row_stride, w, out, out_row_stride, static_cast<cudaStream_t>(stream), -1);
}

extern "C" dd_status dd_forward_host(dd_plan_t plan, const void* host_in, int64_t in_row_stride,
                                     const float* host_w, void* host_out, int64_t out_row_stride, void* stream) {
  NvtxRange range("dd_forward_host");
  clear_error();
  if (!plan || !host_in || !host_out) return set_error(DD_ERR_ARG, "dd_forward_host: NULL argument");
  if (in_row_stride < plan->n_in) return set_error(DD_ERR_SHAPE, "dd_forward_host: in_row_stride < n_in");
  if (out_row_stride < plan->n_out) return set_error(DD_ERR_SHAPE, "dd_forward_host: out_row_stride < n_out");
  if (plan->dtype == DD_U8_I32 && host_w)
    return set_error(DD_ERR_UNSUPPORTED, "dd_forward_host: uint8 plans take unit weights only");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t elem = plan->dtype == DD_U8_I32 ? 1 : 4;
  // device rows padded so that every configuration applies
  const int64_t dev_in_stride = plan_in_stride(*plan);
  const size_t in_bytes = (size_t)plan->C * dev_in_stride * elem;
  const size_t out_bytes = (size_t)plan->n_dm * plan->n_out * 4;
  if (plan->h_in_bytes < in_bytes) {
    cudaFree(plan->h_dev_in);
    plan->h_dev_in = nullptr;
    plan->h_in_bytes = 0;
    if (cudaMalloc(&plan->h_dev_in, in_bytes) != cudaSuccess)
      return set_error(DD_ERR_NOMEM, "dd_forward_host: cannot allocate %zu input bytes", in_bytes);
    plan->h_in_bytes = in_bytes;
  }
  if (plan->h_out_bytes < out_bytes) {
    cudaFree(plan->h_dev_out);
    plan->h_dev_out = nullptr;
    plan->h_out_bytes = 0;
    if (cudaMalloc(&plan->h_dev_out, out_bytes) != cudaSuccess)
      return set_error(DD_ERR_NOMEM, "dd_forward_host: cannot allocate %zu output bytes", out_bytes);
    plan->h_out_bytes = out_bytes;
  }
  if (host_w && !plan->h_dev_w) {
    if (cudaMalloc(&plan->h_dev_w, (size_t)plan->C * sizeof(float)) != cudaSuccess)
      return set_error(DD_ERR_NOMEM, "dd_forward_host: cannot allocate weights");
  }
  // The output runs in up to three time chunks as a pipeline on plan-owned
  // streams: the copy-in of the input columns chunk k needs beyond those
  // already on the device, chunk k's kernel, and chunk k's copy-out.
  // A short first chunk lets the kernels start early, a short last chunk lets
  // the copy-out finish soon after them, and the middle chunk keeps the
  // kernel's grid large; the copies of the other chunks overlap the kernels.
  // Each output element is computed as in one launch: the result is
  // bit-identical.  Chunk edges are multiples of 4096 samples.
  constexpr int64_t kEdge = 4096;
  int64_t edges[4] = {0, plan->n_out, plan->n_out, plan->n_out};
  int n_chunks = 1;
  if (plan->n_out > 3 * kEdge) {
    const int64_t last = plan->n_out - (plan->n_out - 1) / kEdge * kEdge;  // 1..4096
    edges[1] = kEdge;
    edges[2] = plan->n_out - last;
    edges[3] = plan->n_out;
    n_chunks = 3;
  }
  cudaError_t e = cudaSuccess;
  if (!plan->h_streams[0]) {
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
      e = cudaStreamCreateWithFlags(&plan->h_streams[k], cudaStreamNonBlocking);
    if (e != cudaSuccess) return set_cuda_error("dd_forward_host: streams", e);
  }
  while ((int)plan->h_events.size() < 2 * n_chunks + 2) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return set_cuda_error("dd_forward_host: events", e);
    plan->h_events.push_back(ev);
  }
  // chunks alternate between two kernel streams (and two copy-out streams),
  // so a short chunk's blocks fill the last wave of its neighbour's
  cudaStream_t s_in = plan->h_streams[0];
  cudaStream_t s_run[2] = {plan->h_streams[1], plan->h_streams[2]}, s_out[2] = {plan->h_streams[3], plan->h_streams[4]};
  cudaEvent_t ev_fork = plan->h_events[0];
  e = cudaEventRecord(ev_fork, s);  // after the caller's earlier work on `stream`
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ev_fork, 0);
  if (e == cudaSuccess && host_w)
    e = cudaMemcpyAsync(plan->h_dev_w, host_w, plan->C * sizeof(float), cudaMemcpyHostToDevice, s_in);
  if (e != cudaSuccess) return set_cuda_error("dd_forward_host: copy in", e);
  int64_t have = 0;  // input columns already copied
  for (int k = 0; k < n_chunks; ++k) {
    const int64_t t0 = edges[k], t1 = edges[k + 1];
    const int64_t need = t1 + plan->max_delay;
    cudaEvent_t ev_in = plan->h_events[2 + 2 * k], ev_run = plan->h_events[3 + 2 * k];
    e = cudaMemcpy2DAsync(static_cast<unsigned char*>(plan->h_dev_in) + have * elem, dev_in_stride * elem,
                          static_cast<const unsigned char*>(host_in) + have * elem, in_row_stride * elem,
                          (need - have) * elem, plan->C, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_run[k & 1], ev_in, 0);
    if (e != cudaSuccess) return set_cuda_error("dd_forward_host: copy in", e);
    have = need;
    const dd_status st = launch_range(plan, plan->h_dev_in, dev_in_stride, host_w ? plan->h_dev_w : nullptr,
                                      plan->h_dev_out, plan->n_out, t0, t1, s_run[k & 1], -1);
    if (st != DD_OK) return st;
    e = cudaEventRecord(ev_run, s_run[k & 1]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out[k & 1], ev_run, 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(static_cast<unsigned char*>(host_out) + t0 * 4, out_row_stride * 4,
                            static_cast<unsigned char*>(plan->h_dev_out) + t0 * 4, plan->n_out * 4, (t1 - t0) * 4,
                            plan->n_dm, cudaMemcpyDeviceToHost, s_out[k & 1]);
    if (e != cudaSuccess) return set_cuda_error("dd_forward_host: copy out", e);
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {  // join both copy-out streams
    e = cudaEventRecord(plan->h_events[1 - k], s_out[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->h_events[1 - k], 0);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_cuda_error("dd_forward_host: synchronize", e);
  return DD_OK;
}
