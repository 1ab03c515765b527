// Forward dedispersion kernels (Algorithm 1, Section 2.1) for sm_103a.
//
//   out[i][t] = sum_c w[c] * in[c][t + delay(c, i)]
//
// NAIVE  - one output sample per thread and one DM per block row, delays and
//          samples read straight from global memory.  This is the paper's
//          "generically tuned" layout (Section 5) and also the fallback for
//          inputs whose alignment the bulk copies cannot take.
// STAGED - a block owns BD DM trials x BT samples (Section 2.2's 2-D work
//          groups).  For every channel the block needs input samples
//          [t0 + delay(c, i0), t0 + BT + delay(c, i0 + BD - 1)); one 1-D bulk
//          copy per channel moves that span into shared memory, where it
//          serves all BD trials.  Channel chunks flow through a STAGES-deep
//          mbarrier pipeline so copies overlap the sums.  Each thread keeps
//          (BD/8) x (BT/32) sums in registers; lanes run along time so shared
//          reads and global writes are contiguous across the warp.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"
#include "ptx.cuh"

namespace dd {

template <typename Tin>
struct AccOf;
template <>
struct AccOf<float> {
  using type = float;
};
template <>
struct AccOf<uint8_t> {
  using type = int32_t;
};

// ------------------------------------------------------------------ NAIVE

template <typename Tin, bool WEIGHTED>
__global__ void __launch_bounds__(256) fwd_naive_kernel(FwdArgs a) {
  using Tacc = typename AccOf<Tin>::type;
  const Tin* __restrict__ in = static_cast<const Tin*>(a.in);
  Tacc* __restrict__ out = static_cast<Tacc*>(a.out);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_out) return;
  for (int64_t i = blockIdx.y; i < a.n_dm; i += gridDim.y) {
    const int32_t* __restrict__ drow = a.delays + i * a.C;
    Tacc acc = 0;
    for (int c = 0; c < a.C; ++c) {
      const Tin v = __ldg(in + (int64_t)c * a.in_stride + t + __ldg(drow + c));
      if constexpr (WEIGHTED) {
        acc = fmaf(__ldg(a.w + c), v, acc);
      } else {
        acc += (Tacc)v;
      }
    }
    out[i * a.out_stride + t] = acc;
  }
}

// ----------------------------------------------------------------- STAGED

// Shared-memory layout of the staged kernels:
//   [STAGES][CC][pitch] input spans (Tin), [STAGES][CC][BD] int32 delay
//   slices, [STAGES] mbarriers.
template <typename Tin>
__host__ __device__ constexpr int staged_smem_bytes(int stages, int cc, int bd, int pitch) {
  return stages * cc * pitch * (int)sizeof(Tin) + stages * cc * bd * 4 + stages * 8;
}

template <typename Tin, bool WEIGHTED, int BD, int BT, int CC, int STAGES>
__global__ void __launch_bounds__(256) fwd_staged_kernel(FwdArgs a, int pitch) {
  using Tacc = typename AccOf<Tin>::type;
  constexpr int V = 16 / (int)sizeof(Tin);  // elements per 16 bytes
  constexpr int NW = 8;
  constexpr int DPW = BD / NW;
  constexpr int SPL = BT / 32;
  static_assert(BD % NW == 0 && BT % 32 == 0 && BD % 4 == 0, "tile shape");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  Tin* sin = reinterpret_cast<Tin*>(smem_raw);
  int32_t* sdel = reinterpret_cast<int32_t*>(smem_raw + (size_t)STAGES * CC * pitch * sizeof(Tin));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sdel + STAGES * CC * BD);

  const Tin* __restrict__ in = static_cast<const Tin*>(a.in);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t t0 = (int64_t)blockIdx.x * BT;
  const int i0 = blockIdx.y * BD;
  const int nt = (int)min((int64_t)BT, a.n_out - t0);
  const int nchunks = (a.C + CC - 1) / CC;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // Producer (thread 0): stage chunk k (channels [k*CC, k*CC + CC)) into stage k % STAGES.
  auto issue = [&](int k) {
    const int s = k % STAGES;
    const int c0 = k * CC;
    const int cn = min(CC, a.C - c0);
    uint32_t bytes = 0;
    for (int j = 0; j < cn; ++j) {
      const int64_t c = c0 + j;
      const int64_t lo = t0 + __ldg(a.delaysT + c * a.n_dm_pad + i0);
      const int64_t hi = t0 + nt + __ldg(a.delaysT + c * a.n_dm_pad + i0 + BD - 1);
      const int64_t al = lo & ~(int64_t)(V - 1);
      const int64_t ah = (hi + V - 1) & ~(int64_t)(V - 1);
      bytes += (uint32_t)((ah - al) * (int64_t)sizeof(Tin)) + BD * 4;
    }
    mbar_arrive_expect_tx(&bars[s], bytes);
    for (int j = 0; j < cn; ++j) {
      const int64_t c = c0 + j;
      const int64_t lo = t0 + __ldg(a.delaysT + c * a.n_dm_pad + i0);
      const int64_t hi = t0 + nt + __ldg(a.delaysT + c * a.n_dm_pad + i0 + BD - 1);
      const int64_t al = lo & ~(int64_t)(V - 1);
      const int64_t ah = (hi + V - 1) & ~(int64_t)(V - 1);
      bulk_g2s(sin + (size_t)(s * CC + j) * pitch, in + c * a.in_stride + al,
               (uint32_t)((ah - al) * (int64_t)sizeof(Tin)), &bars[s]);
      bulk_g2s(sdel + (s * CC + j) * BD, a.delaysT + c * a.n_dm_pad + i0, BD * 4, &bars[s]);
    }
  };

  if (tid == 0) {
    for (int k = 0; k < min(STAGES, nchunks); ++k) issue(k);
  }

  Tacc acc[DPW][SPL];
#pragma unroll
  for (int m = 0; m < DPW; ++m)
#pragma unroll
    for (int q = 0; q < SPL; ++q) acc[m][q] = 0;

  for (int k = 0; k < nchunks; ++k) {
    const int s = k % STAGES;
    const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k / STAGES) & 1), kWaitLimitCycles);
    // The barrier also tells every thread that chunk k-1 is fully consumed.
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        report_error(a.status, kDevWaitTimeout);
        // let copies already in flight land before the block exits
        for (int kk = k; kk < min(k + STAGES, nchunks); ++kk)
          (void)mbar_wait_bounded(&bars[kk % STAGES], (uint32_t)((kk / STAGES) & 1), kWaitLimitCycles);
      }
      return;
    }
    if (tid == 0 && k >= 1 && k - 1 + STAGES < nchunks) issue(k - 1 + STAGES);

    const int c0 = k * CC;
    const int cn = min(CC, a.C - c0);
    for (int j = 0; j < cn; ++j) {
      const Tin* row = sin + (size_t)(s * CC + j) * pitch;
      const int32_t* dl = sdel + (s * CC + j) * BD;
      const int d0 = dl[0];
      const int64_t al = (t0 + d0) & ~(int64_t)(V - 1);
      const int base = (int)(t0 + d0 - al);  // row index of (DM i0, sample t0)
      float wc = 1.0f;
      if constexpr (WEIGHTED) wc = __ldg(a.w + c0 + j);
#pragma unroll
      for (int m = 0; m < DPW; ++m) {
        const int off = base + dl[warp + m * NW] - d0 + lane;
#pragma unroll
        for (int q = 0; q < SPL; ++q) {
          const Tin v = row[off + 32 * q];
          if constexpr (WEIGHTED) {
            acc[m][q] = fmaf(wc, v, acc[m][q]);
          } else {
            acc[m][q] += (Tacc)v;
          }
        }
      }
    }
  }

  Tacc* __restrict__ out = static_cast<Tacc*>(a.out);
#pragma unroll
  for (int m = 0; m < DPW; ++m) {
    const int i = i0 + warp + m * NW;
    if (i < a.n_dm) {
#pragma unroll
      for (int q = 0; q < SPL; ++q) {
        const int tt = lane + 32 * q;
        if (tt < nt) out[(int64_t)i * a.out_stride + t0 + tt] = acc[m][q];
      }
    }
  }
}

// --------------------------------------------------------------- dispatch

template <typename Tin, bool WEIGHTED>
static cudaError_t launch_naive(const TileConfig& cfg, const FwdArgs& a, cudaStream_t s) {
  dim3 block(cfg.threads);
  dim3 grid((unsigned)((a.n_out + cfg.threads - 1) / cfg.threads), (unsigned)min(a.n_dm, 65535));
  fwd_naive_kernel<Tin, WEIGHTED><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename Tin, bool WEIGHTED, int BD, int BT, int CC, int STAGES>
static cudaError_t launch_staged_t(const TileConfig& cfg, const FwdArgs& a, cudaStream_t s) {
  auto kern = fwd_staged_kernel<Tin, WEIGHTED, BD, BT, CC, STAGES>;
  const int smem = staged_smem_bytes<Tin>(STAGES, CC, BD, cfg.pitch);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((a.n_out + BT - 1) / BT), (unsigned)((a.n_dm + BD - 1) / BD));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  kern<<<grid, 256, smem, s>>>(a, cfg.pitch);
  return cudaGetLastError();
}

#define DD_STAGED_CASES(X)   \
  X(8, 256, 8, 3)            \
  X(16, 256, 8, 3)           \
  X(32, 256, 8, 3)           \
  X(16, 512, 8, 3)           \
  X(8, 512, 8, 3)            \
  X(8, 1024, 4, 3)           \
  X(32, 512, 4, 3)           \
  X(64, 256, 4, 3)

template <typename Tin, bool WEIGHTED>
static cudaError_t launch_staged(const TileConfig& cfg, const FwdArgs& a, cudaStream_t s) {
#define X(BD_, BT_, CC_, ST_)                                                    \
  if (cfg.bd == BD_ && cfg.bt == BT_ && cfg.cc == CC_ && cfg.stages == ST_) \
    return launch_staged_t<Tin, WEIGHTED, BD_, BT_, CC_, ST_>(cfg, a, s);
  DD_STAGED_CASES(X)
#undef X
  return cudaErrorInvalidConfiguration;
}

cudaError_t launch_regwin(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s);

cudaError_t launch_forward(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s) {
  const bool weighted = a.w != nullptr;
  switch (cfg.kind) {
    case Kind::Naive:
      if (dtype == DD_U8_I32) return launch_naive<uint8_t, false>(cfg, a, s);
      return weighted ? launch_naive<float, true>(cfg, a, s) : launch_naive<float, false>(cfg, a, s);
    case Kind::Staged:
      if (dtype == DD_U8_I32) return launch_staged<uint8_t, false>(cfg, a, s);
      return weighted ? launch_staged<float, true>(cfg, a, s) : launch_staged<float, false>(cfg, a, s);
    case Kind::RegWin:
      return launch_regwin(cfg, dtype, a, s);
  }
  return cudaErrorInvalidConfiguration;
}

std::vector<TileConfig> staged_menu(dd_dtype dtype) {
  std::vector<TileConfig> v;
  (void)dtype;
  v.push_back({Kind::Naive, 1, 256, 0, 0, 256, 0, 0, 0, "naive_t256"});
  v.push_back({Kind::Naive, 1, 128, 0, 0, 128, 0, 0, 0, "naive_t128"});
#define X(BD_, BT_, CC_, ST_)                                                            \
  v.push_back({Kind::Staged, BD_, BT_, CC_, ST_, 256, 0, 0, 0,                           \
               "staged_d" #BD_ "_t" #BT_ "_c" #CC_ "_s" #ST_});
  DD_STAGED_CASES(X)
#undef X
  return v;
}

int staged_smem_for(dd_dtype dtype, int stages, int cc, int bd, int pitch) {
  return dtype == DD_U8_I32 ? staged_smem_bytes<uint8_t>(stages, cc, bd, pitch)
                            : staged_smem_bytes<float>(stages, cc, bd, pitch);
}

}  // namespace dd
