// Adjoint (transpose) of Algorithm 1 and the per-channel weight gradient.
//
// Algorithm 1 reads in[c][t + d(c,i)] for every (i, t, c), so its transpose
// sends grad_out[i][t] back to that position:
//   G[c][u] = sum over i with 0 <= u - d(c,i) < n_out of grad_out[i][u - d(c,i)].
// Writing P[i][v] = grad_out[i][v - max_d] (zero outside [max_d, max_d + n_out))
// turns this into another shifted sum over a reduction index:
//   G[c][u] = sum_i P[i][u + (max_d - d(c,i))],
// i.e. Algorithm 1 with the roles of channel and DM trial swapped and delays
// max_d - d(c,i) >= 0, which grow with c because d(c,i) shrinks with frequency.
// The adjoint therefore runs on the same tuned forward kernels through a
// transposed plan built on first use, after one zero-padded copy of grad_out.
//   grad_in[c][u] = w[c] * G[c][u]
//   grad_w[c]     = sum_i sum_t grad_out[i][t] in[c][t + d(c,i)] = sum_u in[c][u] G[c][u]
// The weight gradient is one dot product per channel, reduced in a fixed
// order (deterministic, no atomics).  Requested alone, on plans and inputs
// the 9-trial Tensor-Memory forward takes, it is computed directly on that
// kernel's tiles instead (fwd_tmw9.cu), again in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "dd_errors.h"
#include "dd_internal.h"

namespace dd {

static dd_status adjoint_plan(dd_plan_s* p, dd_plan_s** out) {
  if (p->adj) {
    *out = p->adj;
    return DD_OK;
  }
  dd_plan_s* q = new (std::nothrow) dd_plan_s();
  if (!q) return set_error(DD_ERR_NOMEM, "dd_adjoint: host allocation failed");
  q->C = p->n_dm;
  q->n_dm = p->C;
  q->n_out = p->n_in;
  q->dtype = DD_F32_F32;
  q->f_low = p->f_low;
  q->chan_bw = p->chan_bw;
  q->t_samp = p->t_samp;
  q->delays.resize((size_t)p->C * p->n_dm);
  for (int32_t c = 0; c < p->C; ++c)
    for (int32_t i = 0; i < p->n_dm; ++i)
      q->delays[(size_t)c * p->n_dm + i] = p->max_delay - p->delays[(size_t)i * p->C + c];
  dd_status st = finish_plan(q);
  if (st != DD_OK) {
    delete q;
    return st;
  }
  p->adj = q;
  *out = q;
  return DD_OK;
}

// grad_w[c] = sum_u in[c][u] * g[c][u]: one block per channel, double sums,
// fixed reduction tree.
__global__ void __launch_bounds__(256) wgrad_dot_kernel(const float* __restrict__ in, int64_t in_stride,
                                                        const float* __restrict__ g, int64_t g_stride, int64_t n,
                                                        float* __restrict__ grad_w) {
  const int c = blockIdx.x;
  const float* a = in + (int64_t)c * in_stride;
  const float* b = g + (int64_t)c * g_stride;
  double acc = 0.0;
  for (int64_t u = threadIdx.x; u < n; u += blockDim.x) acc += (double)__ldg(a + u) * (double)__ldg(b + u);
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad_w[c] = (float)red[0];
}

// rows[c][u] *= w[c] for u < n
__global__ void scale_rows_kernel(float* __restrict__ rows, int64_t stride, int64_t n, const float* __restrict__ w) {
  const int c = blockIdx.y;
  const float wc = __ldg(w + c);
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    rows[(int64_t)c * stride + u] *= wc;
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_adjoint(dd_plan_t plan, const float* grad_out, int64_t go_row_stride, const float* w,
                                float* grad_in, int64_t gi_row_stride, const float* in, int64_t in_row_stride,
                                float* grad_w, void* stream) {
  NvtxRange range("dd_adjoint");
  clear_error();
  if (!plan) return set_error(DD_ERR_ARG, "dd_adjoint: plan is NULL");
  if (plan->dtype != DD_F32_F32) return set_error(DD_ERR_UNSUPPORTED, "dd_adjoint: float32 plans only");
  if (!grad_out) return set_error(DD_ERR_ARG, "dd_adjoint: grad_out is NULL");
  if (!grad_in && !grad_w) return set_error(DD_ERR_ARG, "dd_adjoint: neither grad_in nor grad_w requested");
  if (grad_w && !in) return set_error(DD_ERR_ARG, "dd_adjoint: grad_w needs the forward input");
  if (go_row_stride < plan->n_out) return set_error(DD_ERR_SHAPE, "dd_adjoint: go_row_stride < n_out");
  if (grad_in && gi_row_stride < plan->n_in) return set_error(DD_ERR_SHAPE, "dd_adjoint: gi_row_stride < n_in");
  if (grad_w && in_row_stride < plan->n_in) return set_error(DD_ERR_SHAPE, "dd_adjoint: in_row_stride < n_in");
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // The weight gradient alone, on a plan and input layout the 9-trial
  // Tensor-Memory forward takes: the forward's own tiles multiply grad_out
  // with the input windows (about one forward's time, no transposed plan).
  if (grad_w && !grad_in) {
    const FwdArgs a = plan_args(plan, in, in_row_stride, nullptr, nullptr, 0, 0, plan->n_out);
    const int64_t n = tmw9_wgrad_partials(a);
    // (12 partial sums per channel and tile: past 1 GiB of them, as for very
    // long outputs, the transposed path below needs less memory)
    if (n > 0 && n <= ((int64_t)1 << 28)) {
      if (plan->adj_wpart_floats < n) {
        cudaFree(plan->adj_wpart);
        plan->adj_wpart_floats = 0;
        if (cudaMalloc(&plan->adj_wpart, (size_t)n * sizeof(float)) != cudaSuccess) {
          plan->adj_wpart = nullptr;
          return set_error(DD_ERR_NOMEM, "dd_adjoint: cannot allocate %lld floats of partial sums", (long long)n);
        }
        plan->adj_wpart_floats = n;
      }
      const cudaError_t e = launch_tmw9_wgrad(a, grad_out, go_row_stride, plan->adj_wpart, grad_w, s);
      if (e != cudaSuccess) return set_cuda_error("dd_adjoint: weight gradient", e);
      return DD_OK;
    }
  }

  dd_plan_s* q = nullptr;
  dd_status st = adjoint_plan(plan, &q);
  if (st != DD_OK) return st;

  // zero-padded copy of grad_out: P[i][max_d + t] = grad_out[i][t]
  if (!plan->adj_pad) {
    const int64_t stride = plan_in_stride(*q);  // the transposed plan's kernels take it at full speed
    const size_t bytes = (size_t)plan->n_dm * stride * sizeof(float);
    if (cudaMalloc(&plan->adj_pad, bytes) != cudaSuccess) {
      plan->adj_pad = nullptr;
      return set_error(DD_ERR_NOMEM, "dd_adjoint: cannot allocate %zu bytes of padded grad_out", bytes);
    }
    plan->adj_pad_stride = stride;
    cudaError_t e = cudaMemsetAsync(plan->adj_pad, 0, bytes, s);  // pads stay zero from here on
    if (e != cudaSuccess) return set_cuda_error("dd_adjoint: memset", e);
  }
  cudaError_t e = cudaMemcpy2DAsync(plan->adj_pad + plan->max_delay, plan->adj_pad_stride * sizeof(float), grad_out,
                                    go_row_stride * sizeof(float), plan->n_out * sizeof(float), plan->n_dm,
                                    cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return set_cuda_error("dd_adjoint: pad copy", e);

  float* g = grad_in;
  int64_t g_stride = gi_row_stride;
  if (!g) {
    if (!plan->adj_g) {
      const int64_t stride = (plan->n_in + 3) / 4 * 4;
      const size_t bytes = (size_t)plan->C * stride * sizeof(float);
      if (cudaMalloc(&plan->adj_g, bytes) != cudaSuccess) {
        plan->adj_g = nullptr;
        return set_error(DD_ERR_NOMEM, "dd_adjoint: cannot allocate %zu bytes for the transpose", bytes);
      }
      plan->adj_g_stride = stride;
    }
    g = plan->adj_g;
    g_stride = plan->adj_g_stride;
  }
  st = forward_device(q, plan->adj_pad, plan->adj_pad_stride, nullptr, g, g_stride, s, -1);
  if (st != DD_OK) return st;
  if (grad_w) {
    wgrad_dot_kernel<<<plan->C, 256, 0, s>>>(in, in_row_stride, g, g_stride, plan->n_in, grad_w);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error("dd_adjoint: weight gradient", e);
  }
  if (grad_in && w) {
    dim3 grid((unsigned)std::min<int64_t>((plan->n_in + 255) / 256, 1024), (unsigned)plan->C);
    scale_rows_kernel<<<grid, 256, 0, s>>>(grad_in, gi_row_stride, plan->n_in, w);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error("dd_adjoint: weights", e);
  }
  return DD_OK;
}
