// Boxcar-8 S/N detection loss over a dedispersed block, and its gradient.
//
// Not part of the paper: this is the loss of the differentiable
// configuration (dedisperse -> 8-sample boxcar -> maximum S/N).  Per row i:
// b[t] = sum_{k<8} x[i][t+k], mean m and population sd s of b over
// t < nb = n_cols - 7, z[t] = (b[t] - m) / s.  loss = -max_{i,t} z (first on
// ties).  For the best row i*, t*:
//   d z[t*] / d b[t] = ((t == t*) - 1/nb) / s - z[t*] z[t] / (nb s)
//   d loss / d x[i*][u] = -sum over t in [u-7, u] of d z[t*] / d b[t].
// Each thread sums in two-float arithmetic (about 48 bits), each block in
// double; each row is one block with a fixed reduction tree.
#include <cuda_runtime.h>

#include <cfloat>
#include <mutex>

#include "dd_errors.h"
#include "dd_internal.h"

namespace dd {

constexpr int kBox = 8;

struct RowStat {
  double z;      // best S/N in the row (-inf if the row is constant)
  double mean;
  double sd;
  int64_t t;     // boxcar start of the best S/N
};

__device__ __forceinline__ double boxcar(const float* row, int64_t t) {
  double b = 0.0;
#pragma unroll
  for (int k = 0; k < kBox; ++k) b += (double)__ldg(row + t + k);
  return b;
}

template <int NT>
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Two-float ("double-float") numbers: h + l with |l| <= ulp(h) / 2, about 48
// significant bits.  Double arithmetic is slow on this GPU's SMs; these
// sums use a few single-precision operations each (Knuth's two-sum, Dekker's
// fast two-sum and an FMA-based exact product), with explicit round-to-nearest
// intrinsics so that the compiler neither fuses nor reorders them.
struct DF {
  float h, l;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add_f(DF a, float b) {
  const DF s = two_sum(a.h, b);
  return fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.h, b.h);
  const DF t = two_sum(a.l, b.l);
  const DF u = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(u.h, __fadd_rn(u.l, t.l));
}

// d * d for a two-float d, as a two-float (the low part's square is dropped)
__device__ __forceinline__ DF df_sqr(DF d) {
  const float p = __fmul_rn(d.h, d.h);
  const float e = __fmaf_rn(d.h, d.h, -p);
  return fast_two_sum(p, __fmaf_rn(__fmul_rn(2.0f, d.h), d.l, e));
}

__device__ __forceinline__ DF df_of(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_value(DF a) { return (double)a.h + (double)a.l; }

// a > b for normalised two-floats
__device__ __forceinline__ bool df_gt(DF a, DF b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

// The boxcar starting at t as a two-float (exact while the 8 values' nonzero
// magnitudes lie within a factor of about 2^21: 48 bits hold the sum of eight
// 24-bit significands spread that far).
__device__ __forceinline__ DF boxcar_df(const float* row, int64_t t) {
  DF b{0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < kBox; ++k) b = df_add_f(b, __ldg(row + t + k));
  return b;
}

// One block per row: mean, sd, best S/N and where it is.  Thread j takes
// the boxcar starts j, j + NT, ... (coalesced loads; each boxcar summed from
// its 8 values in two-float arithmetic, exact while their nonzero magnitudes
// lie within a factor of about 2^21, so b equals the direct 8-term sum and
// its double value).  Pass 1: the sum of b and the largest b (first t); pass 2: the
// variance about the mean (each thread's sums in two-float, the block's in
// double); the best S/N is (b_max - mean) / sd in double.  S/N is monotonic
// in b, so the first maximum of S/N lies among the starts whose b is within
// rounding of b_max; pass 3 takes the first start before that t whose S/N
// equals the best (a different t only when two sums round to one S/N).
template <int NT>
__global__ void __launch_bounds__(NT) snr_rows_kernel(const float* __restrict__ x, int64_t stride, int64_t n_cols,
                                                      RowStat* __restrict__ stats) {
  __shared__ double red[NT];
  __shared__ double zbest[NT];
  __shared__ int64_t tbest[NT];
  const int i = blockIdx.x;
  const float* row = x + (int64_t)i * stride;
  const int64_t nb = n_cols - kBox + 1;

  // pass 1: sum and largest boxcar
  DF s{0.0f, 0.0f}, bmax{-FLT_MAX, 0.0f};
  int64_t tmax = -1;
  for (int64_t t = threadIdx.x; t < nb; t += NT) {
    const DF b = boxcar_df(row, t);
    s = df_add(s, b);
    if (tmax < 0 || df_gt(b, bmax)) {  // t increases, so the first maximum is kept
      bmax = b;
      tmax = t;
    }
  }
  const double mean = block_sum<NT>(df_value(s), red) / (double)nb;
  zbest[threadIdx.x] = df_value(bmax);
  tbest[threadIdx.x] = tmax;
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      const double bo = zbest[threadIdx.x + h];
      const int64_t to = tbest[threadIdx.x + h];
      if (to >= 0 && (tbest[threadIdx.x] < 0 || bo > zbest[threadIdx.x] ||
                      (bo == zbest[threadIdx.x] && to < tbest[threadIdx.x]))) {
        zbest[threadIdx.x] = bo;
        tbest[threadIdx.x] = to;
      }
    }
    __syncthreads();
  }
  const double b_top = zbest[0];
  const int64_t t_top = tbest[0];
  __syncthreads();

  // pass 2: variance about the mean
  const DF neg_mean = df_of(-mean);
  DF v{0.0f, 0.0f};
  for (int64_t t = threadIdx.x; t < nb; t += NT) v = df_add(v, df_sqr(df_add(boxcar_df(row, t), neg_mean)));
  const double sd = sqrt(block_sum<NT>(df_value(v), red) / (double)nb);
  if (!(sd > 0.0)) {
    if (threadIdx.x == 0) stats[i] = RowStat{-DBL_MAX, mean, sd, -1};
    return;
  }
  const double z_top = (b_top - mean) / sd;

  // pass 3: the first start before t_top with the same S/N, if any
  const double b_cut = b_top - 1e-12 * (fabs(b_top - mean) + fabs(b_top));
  int64_t tf = t_top;
  // below cut_f (two float steps under b_cut) a two-float value is surely below b_cut
  const float cut_f = nextafterf(nextafterf((float)b_cut, -FLT_MAX), -FLT_MAX);
  for (int64_t t = threadIdx.x; t < t_top; t += NT) {
    const DF b = boxcar_df(row, t);
    if (b.h >= cut_f) {
      const double bd = df_value(b);
      if (bd >= b_cut && (bd - mean) / sd == z_top) {
        tf = t;
        break;
      }
    }
  }
  tbest[threadIdx.x] = tf;
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) tbest[threadIdx.x] = min(tbest[threadIdx.x], tbest[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) stats[i] = RowStat{z_top, mean, sd, tbest[0]};
}

// One block: the best row (first on ties) -> result.
template <int NT>
__global__ void __launch_bounds__(NT) snr_pick_kernel(const RowStat* __restrict__ stats, int n_rows,
                                                      dd_snr_result* __restrict__ result) {
  __shared__ double zb[NT];
  __shared__ int ib[NT];
  double z = -DBL_MAX;
  int bi = -1;
  for (int i = threadIdx.x; i < n_rows; i += NT) {
    if (stats[i].t >= 0 && stats[i].z > z) {
      z = stats[i].z;
      bi = i;
    }
  }
  zb[threadIdx.x] = z;
  ib[threadIdx.x] = bi;
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      const double zo = zb[threadIdx.x + h];
      const int io = ib[threadIdx.x + h];
      if (io >= 0 && (ib[threadIdx.x] < 0 || zo > zb[threadIdx.x] || (zo == zb[threadIdx.x] && io < ib[threadIdx.x]))) {
        zb[threadIdx.x] = zo;
        ib[threadIdx.x] = io;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    dd_snr_result r{};
    const int b = ib[0];
    if (b >= 0) {
      r.snr = stats[b].z;
      r.loss = -stats[b].z;
      r.mean = stats[b].mean;
      r.std = stats[b].sd;
      r.best_t = stats[b].t;
      r.best_row = b;
      r.valid = 1;
    } else {
      r.best_row = -1;
      r.best_t = -1;
      r.valid = 0;
    }
    *result = r;
  }
}

// d loss / d x for the best row (the other rows were zeroed by the caller).
__global__ void snr_grad_kernel(const float* __restrict__ x, int64_t stride, int64_t n_cols,
                                const dd_snr_result* __restrict__ result, float* __restrict__ grad,
                                int64_t grad_stride) {
  const dd_snr_result r = *result;
  if (!r.valid) return;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_cols) return;
  const float* row = x + (int64_t)r.best_row * stride;
  const int64_t nb = n_cols - kBox + 1;
  double acc = 0.0;
  const int64_t t_lo = u - (kBox - 1) > 0 ? u - (kBox - 1) : 0;
  const int64_t t_hi = u < nb - 1 ? u : nb - 1;
  for (int64_t t = t_lo; t <= t_hi; ++t) {
    const double z = (boxcar(row, t) - r.mean) / r.std;
    acc += ((t == r.best_t ? 1.0 : 0.0) - 1.0 / (double)nb) / r.std - r.snr * z / ((double)nb * r.std);
  }
  grad[(int64_t)r.best_row * grad_stride + u] = (float)(-acc);
}

dd_status boxcar_snr_launch(const char* who, const float* x, int64_t row_stride, int32_t n_rows, int64_t n_cols,
                            dd_snr_result* result, float* grad, int64_t grad_stride, cudaStream_t s, void* scratch) {
  constexpr int NT = 256;
  RowStat* stats = static_cast<RowStat*>(scratch);
  snr_rows_kernel<NT><<<n_rows, NT, 0, s>>>(x, row_stride, n_cols, stats);
  snr_pick_kernel<NT><<<1, NT, 0, s>>>(stats, n_rows, result);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && grad) {
    e = cudaMemset2DAsync(grad, grad_stride * sizeof(float), 0, n_cols * sizeof(float), n_rows, s);
    if (e == cudaSuccess) {
      snr_grad_kernel<<<(unsigned)((n_cols + 255) / 256), 256, 0, s>>>(x, row_stride, n_cols, result, grad,
                                                                         grad_stride);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return set_error(DD_ERR_CUDA, "%s: launch: %s (%s)", who, cudaGetErrorString(e),
                                         cudaGetErrorName(e));
  return DD_OK;
}

dd_status boxcar_snr_check(const char* who, const float* x, int64_t row_stride, int32_t n_rows, int64_t n_cols,
                           const dd_snr_result* result, const float* grad, int64_t grad_stride) {
  if (!x || !result) return set_error(DD_ERR_ARG, "%s: x/result is NULL", who);
  if (n_rows <= 0) return set_error(DD_ERR_ARG, "%s: n_rows must be > 0", who);
  if (n_cols < kBox) return set_error(DD_ERR_SHAPE, "%s: n_cols must be >= %d", who, kBox);
  if (row_stride < n_cols) return set_error(DD_ERR_SHAPE, "%s: row_stride < n_cols", who);
  if (grad && grad_stride < n_cols) return set_error(DD_ERR_SHAPE, "%s: grad_stride < n_cols", who);
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_boxcar_snr(const float* x, int64_t row_stride, int32_t n_rows, int64_t n_cols,
                                   dd_snr_result* result, float* grad, int64_t grad_stride, void* stream) {
  NvtxRange range("dd_boxcar_snr");
  clear_error();
  dd_status st = boxcar_snr_check("dd_boxcar_snr", x, row_stride, n_rows, n_cols, result, grad, grad_stride);
  if (st != DD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  const size_t bytes = (size_t)n_rows * sizeof(RowStat);
  if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess)
    return set_error(DD_ERR_NOMEM, "dd_boxcar_snr: cannot allocate %zu bytes of scratch", bytes);
  st = boxcar_snr_launch("dd_boxcar_snr", x, row_stride, n_rows, n_cols, result, grad, grad_stride, s, scratch);
  cudaFreeAsync(scratch, s);
  return st;
}

// ------------------------------------------------------ allocation-free form
// Per-row scratch for dd_boxcar_snr_noalloc.  It is part of the library image,
// so each GPU that loads the library carries it (2 MiB) until the process
// exits, and no call ever has to allocate.  Host code cannot use the symbol
// itself as a device address: the address is looked up per device below.
namespace dd {
static __device__ __align__(256) RowStat g_noalloc_rows[DD_NOALLOC_MAX_ROWS];
constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
// per device: the context the address was looked up in, and the address
struct NoAllocSlot {
  void* ctx = nullptr;
  void* addr = nullptr;
};
static NoAllocSlot g_noalloc[kNoAllocMaxDevices];

typedef int (*CtxGetCurrentFn)(void**);
// The driver's cuCtxGetCurrent, looked up once through the runtime.
static CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  return fn;
}

// Device address of g_noalloc_rows on the current device, looked up on the
// first call for that device, and again whenever the device's context has
// changed since (after cudaDeviceReset the array lives in the new context).
static dd_status noalloc_rows(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error("dd_boxcar_snr_noalloc: cudaGetDevice", e);
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return set_error(DD_ERR_UNSUPPORTED, "dd_boxcar_snr_noalloc: device %d is beyond the %d supported", dev,
                     kNoAllocMaxDevices);
  // make sure the device's primary context exists and is current
  e = cudaFree(nullptr);
  if (e != cudaSuccess) return set_cuda_error("dd_boxcar_snr_noalloc: context", e);
  void* ctx = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get || get(&ctx) != 0 || !ctx)
    return set_error(DD_ERR_CUDA, "dd_boxcar_snr_noalloc: cannot read the current context");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocSlot& slot = g_noalloc[dev];
  if (!slot.addr || slot.ctx != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_rows);
    if (e != cudaSuccess || !p) return set_cuda_error("dd_boxcar_snr_noalloc: cudaGetSymbolAddress", e);
    slot.ctx = ctx;
    slot.addr = p;
  }
  *out = slot.addr;
  return DD_OK;
}
}  // namespace dd

extern "C" dd_status dd_boxcar_snr_noalloc(const float* x, int64_t row_stride, int32_t n_rows, int64_t n_cols,
                                           dd_snr_result* result, float* grad, int64_t grad_stride, void* stream) {
  NvtxRange range("dd_boxcar_snr_noalloc");
  clear_error();
  dd_status st = boxcar_snr_check("dd_boxcar_snr_noalloc", x, row_stride, n_rows, n_cols, result, grad, grad_stride);
  if (st != DD_OK) return st;
  if (n_rows > DD_NOALLOC_MAX_ROWS)
    return set_error(DD_ERR_SHAPE, "dd_boxcar_snr_noalloc: %d rows exceed the fixed scratch of %d rows", n_rows,
                     DD_NOALLOC_MAX_ROWS);
  void* rows = nullptr;
  st = noalloc_rows(&rows);
  if (st != DD_OK) return st;
  return boxcar_snr_launch("dd_boxcar_snr_noalloc", x, row_stride, n_rows, n_cols, result, grad, grad_stride,
                           static_cast<cudaStream_t>(stream), rows);
}
