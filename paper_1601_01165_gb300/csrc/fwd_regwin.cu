// REGWIN forward kernel: data reuse across DM trials in registers.
//
// Section 2 notes that nearby DM trials often need the same or nearly the same
// input samples (equal delays for close DMs), and Section 2.2 exploits this
// with several DMs per work group through local memory or cache.  On GB300 the
// shared-memory path delivers 32 words per clock per SM while the FP32 pipes
// retire 128 adds per clock, so one shared load per add caps the kernel at a
// quarter of the add rate.  This kernel moves the reuse one level further in:
//
//  * a warp owns a group of G = 8 consecutive DM trials and 32 * SPL
//    consecutive output samples; lane l owns samples [l*SPL, (l+1)*SPL);
//  * for each channel, the 8 trials of a group need the samples at offsets
//    o_0 = 0 <= o_1 <= ... <= o_7 past the group's first delay (the plan
//    precomputes them per (channel, group) as one 16-byte descriptor);
//  * the lane loads its window of SPL + o_7 consecutive samples from the
//    staged span ONCE into registers and adds win[o_j + q] into the sums of
//    trial j; a warp-uniform switch on o_j selects code whose register
//    indices are static, so the window never leaves registers.
// SPL is odd, so the lanes' windows start in distinct shared-memory banks.
// Staging of the per-channel spans is the same bulk-copy pipeline as the
// STAGED kernel.  At the end the sums are transposed through shared memory
// so global stores are contiguous across the warp.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"
#include "ptx.cuh"

namespace dd {

// Offsets must satisfy o <= kRwMaxOff; the window therefore holds SPL + kRwMaxOff samples.
template <int O, int SPL, bool W>
__device__ __forceinline__ void rw_add(float (&acc)[SPL], const float (&win)[SPL + kRwMaxOff], float wc) {
#pragma unroll
  for (int q = 0; q < SPL; ++q) {
    if constexpr (W) {
      acc[q] = fmaf(wc, win[O + q], acc[q]);
    } else {
      acc[q] += win[O + q];
    }
  }
}

template <int SPL, bool W>
__device__ __forceinline__ void rw_add_switch(int o, float (&acc)[SPL], const float (&win)[SPL + kRwMaxOff],
                                              float wc) {
  switch (o) {
#define DD_RW_CASE(k) \
  case k:             \
    rw_add<k, SPL, W>(acc, win, wc); \
    break;
    DD_RW_CASE(0) DD_RW_CASE(1) DD_RW_CASE(2) DD_RW_CASE(3) DD_RW_CASE(4) DD_RW_CASE(5) DD_RW_CASE(6)
    DD_RW_CASE(7) DD_RW_CASE(8) DD_RW_CASE(9) DD_RW_CASE(10) DD_RW_CASE(11) DD_RW_CASE(12) DD_RW_CASE(13)
    DD_RW_CASE(14) DD_RW_CASE(15) DD_RW_CASE(16) DD_RW_CASE(17) DD_RW_CASE(18) DD_RW_CASE(19)
    DD_RW_CASE(20) DD_RW_CASE(21) DD_RW_CASE(22) DD_RW_CASE(23) DD_RW_CASE(24) DD_RW_CASE(25)
    DD_RW_CASE(26) DD_RW_CASE(27) DD_RW_CASE(28) DD_RW_CASE(29) DD_RW_CASE(30) DD_RW_CASE(31)
#undef DD_RW_CASE
    default:
      break;
  }
}
static_assert(kRwMaxOff == 31, "rw_add_switch enumerates offsets 0..31");

// Load win[0 .. SPL + extra) from row[r0 ...]; extra in [0, kRwMaxOff].
// Entering the fall-through chain at `extra` issues exactly the loads needed.
template <int SPL>
__device__ __forceinline__ void rw_load(float (&win)[SPL + kRwMaxOff], const float* row, int r0, int extra) {
  switch (extra) {
#define DD_RW_LD(k)                        \
  case k:                                  \
    win[SPL + k - 1] = row[r0 + SPL + k - 1]; \
    [[fallthrough]];
    DD_RW_LD(31) DD_RW_LD(30) DD_RW_LD(29) DD_RW_LD(28) DD_RW_LD(27) DD_RW_LD(26) DD_RW_LD(25)
    DD_RW_LD(24) DD_RW_LD(23) DD_RW_LD(22) DD_RW_LD(21) DD_RW_LD(20) DD_RW_LD(19) DD_RW_LD(18)
    DD_RW_LD(17) DD_RW_LD(16) DD_RW_LD(15) DD_RW_LD(14) DD_RW_LD(13) DD_RW_LD(12) DD_RW_LD(11)
    DD_RW_LD(10) DD_RW_LD(9) DD_RW_LD(8) DD_RW_LD(7) DD_RW_LD(6) DD_RW_LD(5) DD_RW_LD(4) DD_RW_LD(3)
    DD_RW_LD(2) DD_RW_LD(1)
#undef DD_RW_LD
    default:
      break;
  }
#pragma unroll
  for (int q = 0; q < SPL; ++q) win[q] = row[r0 + q];
}

// Shared memory: 128 bytes of mbarriers, then [STAGES][CC][pitch] float
// spans and [STAGES][CC][WD] int4 descriptors; the epilogue reuses the area
// after the barriers as [warps][8][32*SPL] float.
constexpr int kRwBarBytes = 128;
__host__ __device__ constexpr int regwin_stage_bytes(int stages, int cc, int wd, int pitch) {
  return kRwBarBytes + stages * cc * pitch * 4 + stages * cc * wd * 16;
}
__host__ __device__ constexpr int regwin_epi_bytes(int wd, int wt, int spl) {
  return kRwBarBytes + wd * wt * kRwGroup * 32 * spl * 4;
}

template <bool WEIGHTED, int WD, int WT, int SPL, int CC, int STAGES>
__global__ void __launch_bounds__(32 * WD * WT, 1) fwd_regwin_f32_kernel(FwdArgs a, int pitch) {
  constexpr int V = 4;
  constexpr int BD = kRwGroup * WD;
  constexpr int BT = 32 * SPL * WT;
  constexpr int NTHR = 32 * WD * WT;
  static_assert(SPL % 2 == 1, "odd samples per lane keep window loads free of bank conflicts");

  static_assert(STAGES * 8 <= kRwBarBytes, "barrier area");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float* sin = reinterpret_cast<float*>(smem_raw + kRwBarBytes);
  int4* sdesc = reinterpret_cast<int4*>(smem_raw + kRwBarBytes + (size_t)STAGES * CC * pitch * 4);

  const float* __restrict__ in = static_cast<const float*>(a.in);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wd = warp % WD, wt = warp / WD;
  const int64_t t0 = (int64_t)blockIdx.x * BT;
  const int i0 = blockIdx.y * BD;
  const int g0 = i0 / kRwGroup;
  const int n_groups = a.n_dm_pad / kRwGroup;
  const int nt = (int)min((int64_t)BT, a.n_out - t0);
  const int nchunks = (a.C + CC - 1) / CC;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto span = [&](int64_t c, int64_t& al, int64_t& ah) {
    const int64_t lo = t0 + __ldg(a.delaysT + c * a.n_dm_pad + i0);
    const int64_t hi = t0 + nt + __ldg(a.delaysT + c * a.n_dm_pad + i0 + BD - 1);
    al = lo & ~(int64_t)(V - 1);
    ah = (hi + V - 1) & ~(int64_t)(V - 1);
  };
  auto issue = [&](int k) {
    const int s = k % STAGES;
    const int c0 = k * CC;
    const int cn = min(CC, a.C - c0);
    uint32_t bytes = 0;
    for (int j = 0; j < cn; ++j) {
      int64_t al, ah;
      span(c0 + j, al, ah);
      bytes += (uint32_t)((ah - al) * 4) + WD * 16;
    }
    mbar_arrive_expect_tx(&bars[s], bytes);
    for (int j = 0; j < cn; ++j) {
      const int64_t c = c0 + j;
      int64_t al, ah;
      span(c, al, ah);
      bulk_g2s(sin + (size_t)(s * CC + j) * pitch, in + c * a.in_stride + al, (uint32_t)((ah - al) * 4), &bars[s]);
      bulk_g2s(sdesc + (s * CC + j) * WD, a.regwin_desc + c * n_groups + g0, WD * 16, &bars[s]);
    }
  };

  if (tid == 0) {
    for (int k = 0; k < min(STAGES, nchunks); ++k) issue(k);
  }

  float acc[kRwGroup][SPL];
#pragma unroll
  for (int j = 0; j < kRwGroup; ++j)
#pragma unroll
    for (int q = 0; q < SPL; ++q) acc[j][q] = 0.0f;
  float win[SPL + kRwMaxOff];
#pragma unroll
  for (int q = 0; q < SPL + kRwMaxOff; ++q) win[q] = 0.0f;

  const int lane_t = wt * 32 * SPL + lane * SPL;  // this lane's first sample within the block

  for (int k = 0; k < nchunks; ++k) {
    const int s = k % STAGES;
    const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k / STAGES) & 1), kWaitLimitCycles);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        report_error(a.status, kDevWaitTimeout);
        for (int kk = k; kk < min(k + STAGES, nchunks); ++kk)
          (void)mbar_wait_bounded(&bars[kk % STAGES], (uint32_t)((kk / STAGES) & 1), kWaitLimitCycles);
      }
      return;
    }
    if (tid == 0 && k >= 1 && k - 1 + STAGES < nchunks) issue(k - 1 + STAGES);

    const int c0 = k * CC;
    const int cn = min(CC, a.C - c0);
    for (int j = 0; j < cn; ++j) {
      const float* row = sin + (size_t)(s * CC + j) * pitch;
      const int4 dblk = sdesc[(s * CC + j) * WD];       // group 0 of the block: x = delay(c, i0)
      const int4 dsc = sdesc[(s * CC + j) * WD + wd];   // this warp's group
      const int64_t al = (t0 + dblk.x) & ~(int64_t)(V - 1);
      const int r0 = (int)(t0 + dsc.x - al) + lane_t;
      float wc = 1.0f;
      if constexpr (WEIGHTED) wc = __ldg(a.w + c0 + j);
      rw_load<SPL>(win, row, r0, dsc.w);
      const uint32_t lo4 = (uint32_t)dsc.y, hi4 = (uint32_t)dsc.z;
      rw_add_switch<SPL, WEIGHTED>((int)(lo4 & 0xff), acc[0], win, wc);
      rw_add_switch<SPL, WEIGHTED>((int)((lo4 >> 8) & 0xff), acc[1], win, wc);
      rw_add_switch<SPL, WEIGHTED>((int)((lo4 >> 16) & 0xff), acc[2], win, wc);
      rw_add_switch<SPL, WEIGHTED>((int)(lo4 >> 24), acc[3], win, wc);
      rw_add_switch<SPL, WEIGHTED>((int)(hi4 & 0xff), acc[4], win, wc);
      rw_add_switch<SPL, WEIGHTED>((int)((hi4 >> 8) & 0xff), acc[5], win, wc);
      rw_add_switch<SPL, WEIGHTED>((int)((hi4 >> 16) & 0xff), acc[6], win, wc);
      rw_add_switch<SPL, WEIGHTED>((int)(hi4 >> 24), acc[7], win, wc);
    }
  }

  // Epilogue: every stage has been consumed (the last barrier wait covered the
  // last chunk's copies); reuse the span area to transpose the sums.
  __syncthreads();
  float* epi = reinterpret_cast<float*>(smem_raw + kRwBarBytes) + (size_t)warp * kRwGroup * 32 * SPL;
#pragma unroll
  for (int j = 0; j < kRwGroup; ++j)
#pragma unroll
    for (int q = 0; q < SPL; ++q) epi[j * 32 * SPL + lane * SPL + q] = acc[j][q];
  __syncwarp();
  float* __restrict__ out = static_cast<float*>(a.out);
  const int tw0 = wt * 32 * SPL;
  for (int j = 0; j < kRwGroup; ++j) {
    const int i = i0 + wd * kRwGroup + j;
    if (i >= a.n_dm) break;
    float* orow = out + (int64_t)i * a.out_stride + t0 + tw0;
    const int lim = min(32 * SPL, nt - tw0);
    for (int u = lane; u < lim; u += 32) orow[u] = epi[j * 32 * SPL + u];
  }
  (void)NTHR;
}

// ------------------------------------------------------------------ launch

#define DD_REGWIN_CASES(X) \
  X(2, 2, 15, 8, 4)        \
  X(4, 2, 15, 8, 4)        \
  X(4, 1, 15, 8, 4)        \
  X(2, 4, 15, 4, 4)        \
  X(8, 1, 15, 4, 4)        \
  X(4, 2, 11, 8, 4)        \
  X(2, 2, 19, 8, 4)

template <bool W, int WD, int WT, int SPL, int CC, int STAGES>
static cudaError_t launch_rw_t(const TileConfig& cfg, const FwdArgs& a, cudaStream_t s) {
  auto kern = fwd_regwin_f32_kernel<W, WD, WT, SPL, CC, STAGES>;
  const int smem = cfg.smem;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  constexpr int BD = kRwGroup * WD, BT = 32 * SPL * WT;
  dim3 grid((unsigned)((a.n_out + BT - 1) / BT), (unsigned)((a.n_dm + BD - 1) / BD));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  kern<<<grid, 32 * WD * WT, smem, s>>>(a, cfg.pitch);
  return cudaGetLastError();
}

cudaError_t launch_regwin(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s) {
  if (dtype != DD_F32_F32) return cudaErrorInvalidConfiguration;
  const bool w = a.w != nullptr;
#define X(WD_, WT_, SPL_, CC_, ST_)                                                                      \
  if (cfg.bd == kRwGroup * WD_ && cfg.bt == 32 * SPL_ * WT_ && cfg.spl == SPL_ && cfg.cc == CC_ &&     \
      cfg.stages == ST_)                                                                                \
    return w ? launch_rw_t<true, WD_, WT_, SPL_, CC_, ST_>(cfg, a, s)                                   \
             : launch_rw_t<false, WD_, WT_, SPL_, CC_, ST_>(cfg, a, s);
  DD_REGWIN_CASES(X)
#undef X
  return cudaErrorInvalidConfiguration;
}

std::vector<TileConfig> regwin_menu(dd_dtype dtype) {
  std::vector<TileConfig> v;
  if (dtype != DD_F32_F32) return v;
#define X(WD_, WT_, SPL_, CC_, ST_)                                                                \
  v.push_back({Kind::RegWin, kRwGroup * WD_, 32 * SPL_ * WT_, CC_, ST_, 32 * WD_ * WT_, SPL_, 0, 0, \
               "regwin_f32_w" #WD_ "x" #WT_ "_s" #SPL_ "_c" #CC_});
  DD_REGWIN_CASES(X)
#undef X
  return v;
}

int regwin_smem_for(dd_dtype dtype, const TileConfig& cfg, int pitch) {
  (void)dtype;
  const int wd = cfg.bd / kRwGroup, wt = cfg.bt / (32 * cfg.spl);
  const int a = regwin_stage_bytes(cfg.stages, cfg.cc, wd, pitch);
  const int b = regwin_epi_bytes(wd, wt, cfg.spl);
  return a > b ? a : b;
}

}  // namespace dd
