// Streaming dedispersion with the max-delay overlap kept on the device.
//
// Section 4.2's real-time criterion is to dedisperse each second of data in
// under a second; Section 2.1 notes that producing s output samples needs
// s + max_delay input samples.  A stream therefore keeps the last max_delay
// samples of every channel on the device: chunk k is copied behind that
// tail, the forward kernel (the plan's tuned configuration, n_out =
// chunk_len) produces chunk_len outputs starting at absolute time
// k*chunk_len - max_delay, and the last max_delay input samples become the
// next tail.  Two buffers alternate so the tail never overlaps its source.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "dd_errors.h"
#include "dd_internal.h"

struct dd_stream_s {
  dd_plan_t chunk_plan = nullptr;  // same geometry, n_out = chunk length
  int64_t n = 0;                   // chunk length
  int32_t max_d = 0;
  int32_t C = 0;
  int elem = 4;
  int64_t stride = 0;              // elements per buffer row (>= max_d + n, the chunk plan's input stride)
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  int64_t pushed = 0;
};

using namespace dd;

static void free_stream(dd_stream_s* st) {
  cudaFree(st->buf[0]);
  cudaFree(st->buf[1]);
  if (st->chunk_plan) dd_plan_destroy(st->chunk_plan);
}

extern "C" dd_status dd_stream_create(dd_stream_t* out, dd_plan_t plan, int64_t chunk_len) {
  clear_error();
  if (!out || !plan || chunk_len <= 0) return set_error(DD_ERR_ARG, "dd_stream_create: bad arguments");
  dd_stream_s* st = new (std::nothrow) dd_stream_s();
  if (!st) return set_error(DD_ERR_NOMEM, "dd_stream_create: host allocation failed");
  dd_status s = dd_plan_dm_range(&st->chunk_plan, plan->C, plan->f_low, plan->chan_bw, plan->t_samp, plan->dm_first,
                                 plan->dm_step, plan->dm_index0, plan->n_dm, chunk_len, plan->dtype);
  if (s != DD_OK) {
    delete st;
    return s;
  }
  // keep the caller's kernel choice when the chunk geometry allows it
  const std::string& want = plan->configs[plan->selected].name;
  for (size_t k = 0; k < st->chunk_plan->configs.size(); ++k)
    if (st->chunk_plan->configs[k].name == want) st->chunk_plan->selected = (int)k;
  st->n = chunk_len;
  st->max_d = plan->max_delay;
  st->C = plan->C;
  st->elem = plan->dtype == DD_U8_I32 ? 1 : 4;
  // rows padded so that every configuration of the chunk plan takes the buffer
  st->stride = plan_in_stride(*st->chunk_plan);
  const size_t bytes = (size_t)stream_buffer_bytes(*st->chunk_plan) / 2;
  cudaError_t e = cudaMalloc(&st->buf[0], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&st->buf[1], bytes);
  if (e == cudaSuccess) e = cudaMemset(st->buf[0], 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(st->buf[1], 0, bytes);
  if (e != cudaSuccess) {
    free_stream(st);
    delete st;
    return set_error(DD_ERR_NOMEM, "dd_stream_create: cannot allocate 2 x %zu bytes of state", bytes);
  }
  *out = st;
  return DD_OK;
}

extern "C" dd_status dd_stream_push(dd_stream_t st, const void* chunk, void* out, int64_t* out_t0, void* stream) {
  NvtxRange range("dd_stream_push");
  clear_error();
  if (!st || !chunk || !out) return set_error(DD_ERR_ARG, "dd_stream_push: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* a = static_cast<char*>(st->buf[st->cur]);
  char* b = static_cast<char*>(st->buf[st->cur ^ 1]);
  const size_t pitch = (size_t)st->stride * st->elem;
  cudaError_t e = cudaMemcpy2DAsync(a + (size_t)st->max_d * st->elem, pitch, chunk, (size_t)st->n * st->elem,
                                    (size_t)st->n * st->elem, st->C, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return set_cuda_error("dd_stream_push: chunk copy", e);
  dd_status r = forward_device(st->chunk_plan, a, st->stride, nullptr, out, st->n, s, -1);
  if (r != DD_OK) return r;
  if (st->max_d > 0) {
    e = cudaMemcpy2DAsync(b, pitch, a + (size_t)st->n * st->elem, pitch, (size_t)st->max_d * st->elem, st->C,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_cuda_error("dd_stream_push: tail copy", e);
  }
  st->cur ^= 1;
  if (out_t0) *out_t0 = st->pushed * st->n - st->max_d;
  ++st->pushed;
  return DD_OK;
}

extern "C" dd_status dd_stream_reset(dd_stream_t st, void* stream) {
  clear_error();
  if (!st) return set_error(DD_ERR_ARG, "dd_stream_reset: NULL stream state");
  // on the caller's stream, so that it is ordered after pushes queued there
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)st->C * st->stride * st->elem;
  cudaError_t e = cudaMemsetAsync(st->buf[0], 0, bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->buf[1], 0, bytes, s);
  if (e != cudaSuccess) return set_cuda_error("dd_stream_reset", e);
  st->cur = 0;
  st->pushed = 0;
  return DD_OK;
}

extern "C" dd_status dd_stream_device_bytes(dd_stream_t st, int64_t* bytes) {
  clear_error();
  if (!st || !bytes) return set_error(DD_ERR_ARG, "dd_stream_device_bytes: NULL argument");
  *bytes = st->chunk_plan->device_bytes + stream_buffer_bytes(*st->chunk_plan);
  return DD_OK;
}

extern "C" dd_status dd_stream_state_bytes(dd_stream_t st, int64_t* bytes) {
  clear_error();
  if (!st || !bytes) return set_error(DD_ERR_ARG, "dd_stream_state_bytes: NULL argument");
  *bytes = (int64_t)st->C * st->max_d * st->elem + (int64_t)sizeof(int64_t);
  return DD_OK;
}

// host layout: int64 chunks pushed, then the tail [C][max_d] of the plan's element type
extern "C" dd_status dd_stream_save(dd_stream_t st, void* host_buf, void* stream) {
  clear_error();
  if (!st || !host_buf) return set_error(DD_ERR_ARG, "dd_stream_save: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::memcpy(host_buf, &st->pushed, sizeof(int64_t));
  if (st->max_d > 0) {
    cudaError_t e = cudaMemcpy2DAsync(static_cast<char*>(host_buf) + sizeof(int64_t), (size_t)st->max_d * st->elem,
                                      st->buf[st->cur], (size_t)st->stride * st->elem, (size_t)st->max_d * st->elem,
                                      st->C, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error("dd_stream_save", e);
  }
  return DD_OK;
}

extern "C" dd_status dd_stream_restore(dd_stream_t st, const void* host_buf, void* stream) {
  clear_error();
  if (!st || !host_buf) return set_error(DD_ERR_ARG, "dd_stream_restore: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t pushed = 0;
  std::memcpy(&pushed, host_buf, sizeof(int64_t));
  if (pushed < 0) return set_error(DD_ERR_ARG, "dd_stream_restore: corrupt state (negative chunk count)");
  if (st->max_d > 0) {
    cudaError_t e = cudaMemcpy2DAsync(st->buf[st->cur], (size_t)st->stride * st->elem,
                                      static_cast<const char*>(host_buf) + sizeof(int64_t),
                                      (size_t)st->max_d * st->elem, (size_t)st->max_d * st->elem, st->C,
                                      cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error("dd_stream_restore", e);
  }
  st->pushed = pushed;
  return DD_OK;
}

extern "C" dd_status dd_stream_destroy(dd_stream_t st) {
  clear_error();
  if (!st) return DD_OK;
  free_stream(st);
  delete st;
  return DD_OK;
}
