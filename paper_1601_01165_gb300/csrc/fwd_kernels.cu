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

// Shared-memory layout of the staged kernels: kStBarBytes of mbarriers, then
// [STAGES][CC][pitch] input spans (Tin) and [STAGES][CC][BD] int32 delay
// slices.  The barriers come first so that a persistent block can work on
// tiles of beams whose pitches differ.
constexpr int kStBarBytes = 128;
template <typename Tin>
__host__ __device__ constexpr int staged_smem_bytes(int stages, int cc, int bd, int pitch) {
  return kStBarBytes + stages * cc * pitch * (int)sizeof(Tin) + stages * cc * bd * 4;
}

__device__ __forceinline__ void init_stage_bars(uint64_t* bars, int stages) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
}

// One tile: DM trials [by*BD, by*BD + BD) x samples [bx*BT, bx*BT + BT).
// `kbase` counts the chunks this block consumed before the tile, so the
// stage barriers' phases carry on across the tiles of a persistent block.
// Returns false (on every thread) if a bounded wait expired.
template <typename Tin, bool WEIGHTED, int BD, int BT, int CC, int STAGES>
__device__ __forceinline__ bool staged_tile(const FwdArgs& a, int pitch, int64_t bx, int by, uint32_t& kbase,
                                            unsigned char* smem_raw) {
  using Tacc = typename AccOf<Tin>::type;
  constexpr int V = 16 / (int)sizeof(Tin);  // elements per 16 bytes
  constexpr int NW = 8;
  constexpr int DPW = BD / NW;
  constexpr int SPL = BT / 32;
  static_assert(BD % NW == 0 && BT % 32 == 0 && BD % 4 == 0, "tile shape");
  static_assert(STAGES * 8 <= kStBarBytes, "barrier area");

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  Tin* sin = reinterpret_cast<Tin*>(smem_raw + kStBarBytes);
  int32_t* sdel = reinterpret_cast<int32_t*>(smem_raw + kStBarBytes + (size_t)STAGES * CC * pitch * sizeof(Tin));

  const Tin* __restrict__ in = static_cast<const Tin*>(a.in);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t t0 = bx * BT;
  const int i0 = by * BD;
  const int nt = (int)min((int64_t)BT, a.n_out - t0);
  const int nchunks = (a.C + CC - 1) / CC;
  const uint32_t kb = kbase;

  // Producer (thread 0): stage chunk k (channels [k*CC, k*CC + CC)) into stage (kb + k) % STAGES.
  auto issue = [&](int k) {
    const int s = (int)((kb + (uint32_t)k) % STAGES);
    const int c0 = k * CC;
    const int cn = min(CC, a.C - c0);
    auto span = [&](int64_t c, int64_t& al, int64_t& ah) {
      const int64_t lo = t0 + __ldg(a.delaysT + c * a.n_dm_pad + i0);
      const int64_t hi = t0 + nt + __ldg(a.delaysT + c * a.n_dm_pad + i0 + BD - 1);
      al = lo & ~(int64_t)(V - 1);
      ah = (hi + V - 1) & ~(int64_t)(V - 1);
      // the span fits its shared-memory row and its input row
      if (!DD_INDEX_OK(a.status, al >= 0 && ah - al <= pitch && ah <= a.in_stride)) ah = al + V;
    };
    uint32_t bytes = 0;
    for (int j = 0; j < cn; ++j) {
      int64_t al, ah;
      span(c0 + j, al, ah);
      bytes += (uint32_t)((ah - al) * (int64_t)sizeof(Tin)) + BD * 4;
    }
    mbar_arrive_expect_tx(&bars[s], bytes);
    for (int j = 0; j < cn; ++j) {
      const int64_t c = c0 + j;
      int64_t al, ah;
      span(c, al, ah);
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
    const uint32_t kg = kb + (uint32_t)k;
    const int s = (int)(kg % STAGES);
    const bool ok = mbar_wait_bounded(&bars[s], (kg / STAGES) & 1u, kWaitLimitCycles);
    // The barrier also tells every thread that chunk k-1 is fully consumed.
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        report_error(a.status, kDevWaitTimeout);
        // let copies already in flight land before the block moves on
        for (int kk = k; kk < min(k + STAGES, nchunks); ++kk)
          (void)mbar_wait_bounded(&bars[(kb + kk) % STAGES], ((kb + kk) / STAGES) & 1u, kWaitLimitCycles);
      }
      return false;
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
      if (!DD_INDEX_OK(a.status, base >= 0 && base + dl[BD - 1] - d0 + BT <= pitch)) continue;
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
  kbase = kb + (uint32_t)nchunks;

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
  return true;
}

template <typename Tin, bool WEIGHTED, int BD, int BT, int CC, int STAGES>
__global__ void __launch_bounds__(256) fwd_staged_kernel(FwdArgs a, int pitch) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  init_stage_bars(reinterpret_cast<uint64_t*>(smem_raw), STAGES);
  uint32_t kbase = 0;
  (void)staged_tile<Tin, WEIGHTED, BD, BT, CC, STAGES>(a, pitch, blockIdx.x, blockIdx.y, kbase, smem_raw);
}

// ------------------------------------------------------------------- U8PK
// uint8 -> int32 with packed 16-bit accumulation.  The block stages byte spans
// exactly like STAGED.  A warp owns DPW DM trials x 32 lanes x 28 samples (7
// words; odd, so the lanes' word loads hit distinct banks).  Per channel and
// trial a lane loads 8 words covering its 28 samples at the trial's delay,
// aligns them with one byte permute whose selector is the same for the whole
// warp (the delay modulo 4), splits each aligned word into its even and odd
// samples as 16-bit lanes, and adds two channels at a time into packed 16-bit
// sums (one 3-input integer add per 4 samples and 2 channels).  256 channels
// of 8-bit samples fit a 16-bit lane exactly (256 * 255 < 65536), so every
// 256 channels the packed sums are added into int32 totals and cleared: the
// result is the exact integer sum.
template <int WD, int WT, int DPW, int CC, int STAGES>
__device__ __forceinline__ bool u8pk_tile(const FwdArgs& a, int pitch, int64_t bx, int by, uint32_t& kbase,
                                          unsigned char* smem_raw) {
  constexpr int V = 16;
  constexpr int NW = WD * WT;
  constexpr int KW = 7;               // words per lane
  constexpr int SPL = 4 * KW;         // samples per lane
  constexpr int BD = WD * DPW;
  constexpr int BT = 32 * SPL * WT;
  static_assert(BD % 4 == 0 && BT % 16 == 0, "tile shape");

  static_assert(STAGES * 8 <= kStBarBytes, "barrier area");
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  uint8_t* sin = smem_raw + kStBarBytes;
  int32_t* sdel = reinterpret_cast<int32_t*>(smem_raw + kStBarBytes + (size_t)STAGES * CC * pitch);

  const uint8_t* __restrict__ in = static_cast<const uint8_t*>(a.in);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wd = warp % WD, wt = warp / WD;
  const int64_t t0 = bx * BT;
  const int i0 = by * BD;
  const int nt = (int)min((int64_t)BT, a.n_out - t0);
  const int nchunks = (a.C + CC - 1) / CC;
  const uint32_t kb = kbase;

  auto issue = [&](int k) {
    const int s = (int)((kb + (uint32_t)k) % STAGES);
    const int c0 = k * CC;
    const int cn = min(CC, a.C - c0);
    auto span = [&](int64_t c, int64_t& al, int64_t& ah) {
      const int64_t lo = t0 + __ldg(a.delaysT + c * a.n_dm_pad + i0);
      const int64_t hi = t0 + nt + __ldg(a.delaysT + c * a.n_dm_pad + i0 + BD - 1);
      al = lo & ~(int64_t)(V - 1);
      ah = (hi + V - 1) & ~(int64_t)(V - 1);
      if (!DD_INDEX_OK(a.status, al >= 0 && ah - al <= pitch && ah <= a.in_stride)) ah = al + V;
    };
    uint32_t bytes = 0;
    for (int j = 0; j < cn; ++j) {
      int64_t al, ah;
      span(c0 + j, al, ah);
      bytes += (uint32_t)(ah - al) + BD * 4;
    }
    mbar_arrive_expect_tx(&bars[s], bytes);
    for (int j = 0; j < cn; ++j) {
      const int64_t c = c0 + j;
      int64_t al, ah;
      span(c, al, ah);
      bulk_g2s(sin + (size_t)(s * CC + j) * pitch, in + c * a.in_stride + al, (uint32_t)(ah - al), &bars[s]);
      bulk_g2s(sdel + (s * CC + j) * BD, a.delaysT + c * a.n_dm_pad + i0, BD * 4, &bars[s]);
    }
  };
  if (tid == 0) {
    for (int k = 0; k < min(STAGES, nchunks); ++k) issue(k);
  }

  uint32_t pe[DPW][KW], po[DPW][KW];  // packed 16-bit sums: even / odd samples of each word
  int32_t tot[DPW][SPL];
#pragma unroll
  for (int m = 0; m < DPW; ++m) {
#pragma unroll
    for (int w = 0; w < KW; ++w) pe[m][w] = po[m][w] = 0u;
#pragma unroll
    for (int q = 0; q < SPL; ++q) tot[m][q] = 0;
  }
  auto flush = [&]() {
#pragma unroll
    for (int m = 0; m < DPW; ++m)
#pragma unroll
      for (int w = 0; w < KW; ++w) {
        tot[m][4 * w + 0] += (int32_t)(pe[m][w] & 0xffffu);
        tot[m][4 * w + 2] += (int32_t)(pe[m][w] >> 16);
        tot[m][4 * w + 1] += (int32_t)(po[m][w] & 0xffffu);
        tot[m][4 * w + 3] += (int32_t)(po[m][w] >> 16);
        pe[m][w] = po[m][w] = 0u;
      }
  };
  // aligned words of (trial slot m, channel row j of stage s) -> x[KW]
  auto aligned = [&](int s, int j, int m, uint32_t (&x)[KW]) {
    const uint8_t* row = sin + (size_t)(s * CC + j) * pitch;
    const int32_t* dl = sdel + (s * CC + j) * BD;
    const int d0 = dl[0];
    const int64_t al = (t0 + d0) & ~(int64_t)(V - 1);
    const int off = (int)(t0 + dl[wd * DPW + m] - al) + wt * 32 * SPL + lane * SPL;
    const uint32_t* wp = reinterpret_cast<const uint32_t*>(row) + (off >> 2);
    const uint32_t sel = 0x3210u + 0x1111u * (uint32_t)(off & 3);
    uint32_t wv[KW + 1];
    // the KW + 1 words stay inside the channel's shared-memory row
    if (!DD_INDEX_OK(a.status, off >= 0 && (off >> 2) + KW + 1 <= pitch / 4)) wp = reinterpret_cast<const uint32_t*>(row);
#pragma unroll
    for (int w = 0; w <= KW; ++w) wv[w] = wp[w];
#pragma unroll
    for (int w = 0; w < KW; ++w) x[w] = __byte_perm(wv[w], wv[w + 1], sel);
  };

  int since_flush = 0;
  for (int k = 0; k < nchunks; ++k) {
    const uint32_t kg = kb + (uint32_t)k;
    const int s = (int)(kg % STAGES);
    const bool ok = mbar_wait_bounded(&bars[s], (kg / STAGES) & 1u, kWaitLimitCycles);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        report_error(a.status, kDevWaitTimeout);
        for (int kk = k; kk < min(k + STAGES, nchunks); ++kk)
          (void)mbar_wait_bounded(&bars[(kb + kk) % STAGES], ((kb + kk) / STAGES) & 1u, kWaitLimitCycles);
      }
      return false;
    }
    if (tid == 0 && k >= 1 && k - 1 + STAGES < nchunks) issue(k - 1 + STAGES);
    const int cn = min(CC, a.C - k * CC);
    int j = 0;
    for (; j + 1 < cn; j += 2) {
      if (since_flush >= 255) {  // the next two channels would pass 256
        flush();
        since_flush = 0;
      }
#pragma unroll
      for (int m = 0; m < DPW; ++m) {
        uint32_t x0[KW], x1[KW];
        aligned(s, j, m, x0);
        aligned(s, j + 1, m, x1);
#pragma unroll
        for (int w = 0; w < KW; ++w) {
          pe[m][w] += __byte_perm(x0[w], 0u, 0x4240u) + __byte_perm(x1[w], 0u, 0x4240u);
          po[m][w] += __byte_perm(x0[w], 0u, 0x4341u) + __byte_perm(x1[w], 0u, 0x4341u);
        }
      }
      since_flush += 2;
    }
    if (j < cn) {
      if (since_flush >= 256) {
        flush();
        since_flush = 0;
      }
#pragma unroll
      for (int m = 0; m < DPW; ++m) {
        uint32_t x0[KW];
        aligned(s, j, m, x0);
#pragma unroll
        for (int w = 0; w < KW; ++w) {
          pe[m][w] += __byte_perm(x0[w], 0u, 0x4240u);
          po[m][w] += __byte_perm(x0[w], 0u, 0x4341u);
        }
      }
      since_flush += 1;
    }
  }
  flush();
  kbase = kb + (uint32_t)nchunks;

  // transpose through shared memory (stage area is free: every chunk was consumed)
  __syncthreads();
  int32_t* epi = reinterpret_cast<int32_t*>(smem_raw + kStBarBytes) + (size_t)warp * DPW * 32 * SPL;
#pragma unroll
  for (int m = 0; m < DPW; ++m)
#pragma unroll
    for (int q = 0; q < SPL; ++q) epi[m * 32 * SPL + lane * SPL + q] = tot[m][q];
  __syncwarp();
  int32_t* __restrict__ out = static_cast<int32_t*>(a.out);
  const int tw0 = wt * 32 * SPL;
  const int lim = min(32 * SPL, nt - tw0);
  for (int m = 0; m < DPW; ++m) {
    const int i = i0 + wd * DPW + m;
    if (i >= a.n_dm) break;
    int32_t* orow = out + (int64_t)i * a.out_stride + t0 + tw0;
    for (int u = lane; u < lim; u += 32) orow[u] = epi[m * 32 * SPL + u];
  }
  return true;
}

template <int WD, int WT, int DPW, int CC, int STAGES>
__global__ void __launch_bounds__(32 * WD * WT) fwd_u8pk_kernel(FwdArgs a, int pitch) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  init_stage_bars(reinterpret_cast<uint64_t*>(smem_raw), STAGES);
  uint32_t kbase = 0;
  (void)u8pk_tile<WD, WT, DPW, CC, STAGES>(a, pitch, blockIdx.x, blockIdx.y, kbase, smem_raw);
}

__host__ __device__ constexpr int u8pk_smem_bytes(int stages, int cc, int bd, int pitch, int nw, int dpw) {
  return (stages * cc * pitch + stages * cc * bd * 4) > nw * dpw * 32 * 28 * 4
             ? kStBarBytes + (stages * cc * pitch + stages * cc * bd * 4)
             : kStBarBytes + nw * dpw * 32 * 28 * 4;
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

#define DD_U8PK_CASES(X) \
  X(8, 1, 2, 16, 4)      \
  X(4, 2, 2, 16, 4)      \
  X(8, 1, 4, 16, 3)      \
  X(4, 1, 2, 32, 3)      \
  X(8, 2, 1, 16, 4)

template <int WD, int WT, int DPW, int CC, int ST>
static cudaError_t launch_u8pk_t(const TileConfig& cfg, const FwdArgs& a, cudaStream_t s) {
  auto kern = fwd_u8pk_kernel<WD, WT, DPW, CC, ST>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cfg.smem);
  if (e != cudaSuccess) return e;
  constexpr int BD = WD * DPW, BT = 32 * 28 * WT;
  dim3 grid((unsigned)((a.n_out + BT - 1) / BT), (unsigned)((a.n_dm + BD - 1) / BD));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  kern<<<grid, 32 * WD * WT, cfg.smem, s>>>(a, cfg.pitch);
  return cudaGetLastError();
}

static cudaError_t launch_u8pk(const TileConfig& cfg, const FwdArgs& a, cudaStream_t s) {
#define X(WD_, WT_, DPW_, CC_, ST_)                                                                   \
  if (cfg.bd == WD_ * DPW_ && cfg.bt == 32 * 28 * WT_ && cfg.threads == 32 * WD_ * WT_ && cfg.cc == CC_ && \
      cfg.stages == ST_)                                                                               \
    return launch_u8pk_t<WD_, WT_, DPW_, CC_, ST_>(cfg, a, s);
  DD_U8PK_CASES(X)
#undef X
  return cudaErrorInvalidConfiguration;
}

template <typename Tin, bool WEIGHTED>
static cudaError_t launch_staged(const TileConfig& cfg, const FwdArgs& a, cudaStream_t s) {
#define X(BD_, BT_, CC_, ST_)                                                    \
  if (cfg.bd == BD_ && cfg.bt == BT_ && cfg.cc == CC_ && cfg.stages == ST_) \
    return launch_staged_t<Tin, WEIGHTED, BD_, BT_, CC_, ST_>(cfg, a, s);
  DD_STAGED_CASES(X)
#undef X
  return cudaErrorInvalidConfiguration;
}

cudaError_t launch_tmw6(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s);

cudaError_t launch_forward(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s) {
  const bool weighted = a.w != nullptr;
  switch (cfg.kind) {
    case Kind::Naive:
      if (dtype == DD_U8_I32) return launch_naive<uint8_t, false>(cfg, a, s);
      return weighted ? launch_naive<float, true>(cfg, a, s) : launch_naive<float, false>(cfg, a, s);
    case Kind::Staged:
      if (dtype == DD_U8_I32) return launch_staged<uint8_t, false>(cfg, a, s);
      return weighted ? launch_staged<float, true>(cfg, a, s) : launch_staged<float, false>(cfg, a, s);
    case Kind::TmW6:
      return launch_tmw6(cfg, dtype, a, s);
    case Kind::U8Pk:
      if (dtype != DD_U8_I32 || weighted) return cudaErrorInvalidConfiguration;
      return launch_u8pk(cfg, a, s);
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

std::vector<TileConfig> u8pk_menu(dd_dtype dtype) {
  std::vector<TileConfig> v;
  if (dtype != DD_U8_I32) return v;
#define X(WD_, WT_, DPW_, CC_, ST_)                                                                  \
  v.push_back({Kind::U8Pk, WD_ * DPW_, 32 * 28 * WT_, CC_, ST_, 32 * WD_ * WT_, 28, 0, 0,            \
               "u8pk_w" #WD_ "x" #WT_ "_d" #DPW_ "_c" #CC_ "_st" #ST_});
  DD_U8PK_CASES(X)
#undef X
  return v;
}

int u8pk_smem_for(const TileConfig& cfg, int pitch) {
  const int nw = cfg.threads / 32, wd = nw / (cfg.bt / (32 * 28));
  return u8pk_smem_bytes(cfg.stages, cfg.cc, cfg.bd, pitch, nw, cfg.bd / wd);
}

int staged_smem_for(dd_dtype dtype, int stages, int cc, int bd, int pitch) {
  return dtype == DD_U8_I32 ? staged_smem_bytes<uint8_t>(stages, cc, bd, pitch)
                            : staged_smem_bytes<float>(stages, cc, bd, pitch);
}

}  // namespace dd
