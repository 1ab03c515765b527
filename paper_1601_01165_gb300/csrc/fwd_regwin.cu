// REGWIN forward kernel (float32): data reuse across DM trials in registers.
//
// Section 2 observes that nearby DM trials often need the same input samples
// (equal delays for close DMs) and Section 2.2 turns that into reuse by giving
// a work group several DMs that share loads through local memory or cache.  On
// GB300 the shared-memory path returns 32 words per clock per SM while the FP32
// pipes retire 128 adds per clock, so one shared load per add (the STAGED
// kernel) caps the sums at a quarter of the add rate.  This kernel takes the
// reuse one level further in, to registers:
//
//  * a warp owns a group of G = 8 consecutive DM trials and 32 * SPL
//    consecutive output samples; lane l owns samples [l*SPL, (l+1)*SPL);
//  * for each channel the group's trials need the samples at offsets
//    0 = o_0 <= o_1 <= ... <= o_7 past the group's first delay; the plan stores
//    them per (channel, group) in a 16-byte descriptor;
//  * each lane loads its window of SPL + o_7 consecutive samples from the
//    staged span once, into registers, and adds win[o_j + q] into the sums of
//    trial j.  Register arrays cannot be indexed at run time, so the offset
//    selects straight-line code through one jump-table branch
//    (regwin_dispatch.cuh); the offset is the same for the whole warp, so the
//    branch never diverges.
// SPL is odd, so the lanes' windows start in distinct shared-memory banks.
//
// Staging: lane 0 of warp 0 streams each channel's span of
// [t0 + delay(c, i0), t0 + BT + delay(c, i0 + BD - 1)) into shared memory with
// 1-D bulk copies (STAGES x CC channels in flight).  Full barriers carry the
// copy bytes; empty barriers collect one arrival per warp, so warps drift
// apart by up to STAGES chunks instead of meeting at a block barrier for
// every chunk (only warp 0 waits for the slowest warp before a refill).  A
// separate producer warp would put three warps on one SM sub-partition and
// cap registers at 168, below what the sums and window need.  At the end the sums are transposed through shared memory
// so global stores are contiguous across the warp.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"
#include "ptx.cuh"
#include "regwin_dispatch.cuh"

namespace dd {

static_assert(kRwMaxOff + 1 == kRwDispatchOffsets, "descriptor offsets must match the dispatch table");

// Shared memory: 128 bytes of barriers (full[STAGES], empty[STAGES]), then
// [STAGES][CC][pitch] float spans and [STAGES][CC][WD] int4 descriptors; the
// epilogue reuses the area after the barriers as [consumer warps][8][32*SPL].
constexpr int kRwBarBytes = 128;
__host__ __device__ constexpr int regwin_stage_bytes(int stages, int cc, int wd, int pitch) {
  return kRwBarBytes + stages * cc * pitch * 4 + stages * cc * wd * 16;
}
__host__ __device__ constexpr int regwin_epi_bytes(int wd, int wt, int spl) {
  return kRwBarBytes + wd * wt * kRwGroup * 32 * spl * 4;
}

// Offset k of a packed descriptor word, masked to the dispatch table's range
// (the plan only builds REGWIN descriptors whose offsets are <= 31).
__device__ __forceinline__ uint32_t byte_of(uint32_t v, int k) { return (v >> (8 * k)) & 0x1fu; }

template <bool WEIGHTED, int WD, int WT, int SPL, int CC, int STAGES>
__global__ void __launch_bounds__(32 * WD * WT, 1) fwd_regwin_f32_kernel(FwdArgs a, int pitch) {
  constexpr int V = 4;
  constexpr int BD = kRwGroup * WD;
  constexpr int BT = 32 * SPL * WT;
  constexpr int NCW = WD * WT;  // warps; lane 0 of warp 0 also produces
  constexpr int NWIN = SPL + kRwMaxOff;
  static_assert(SPL % 2 == 1, "odd samples per lane keep window loads free of bank conflicts");
  static_assert(BT % V == 0, "block start must keep 16-byte span alignment arithmetic exact");
  static_assert(2 * STAGES * 8 <= kRwBarBytes, "barrier area");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + STAGES;
  float* sin = reinterpret_cast<float*>(smem_raw + kRwBarBytes);
  int4* sdesc = reinterpret_cast<int4*>(smem_raw + kRwBarBytes + (size_t)STAGES * CC * pitch * 4);
  __shared__ int failed;

  const float* __restrict__ in = static_cast<const float*>(a.in);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t t0 = (int64_t)blockIdx.x * BT;
  const int i0 = blockIdx.y * BD;
  const int g0 = i0 / kRwGroup;
  const int n_groups = a.n_dm_pad / kRwGroup;
  const int nt = (int)min((int64_t)BT, a.n_out - t0);
  const int nchunks = (a.C + CC - 1) / CC;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    failed = 0;
    fence_mbar_init();
  }
  __syncthreads();

  // Producer: lane 0 of warp 0 stages chunk kk (channels [kk*CC, kk*CC + CC))
  // into stage kk % STAGES once every warp has released the chunk that used
  // the stage before.  Returns false if that wait expired.
  auto produce = [&](int kk) -> bool {
    const int s = kk % STAGES;
    if (kk >= STAGES && !mbar_wait_bounded(&empty[s], (uint32_t)(((kk / STAGES) - 1) & 1), kWaitLimitCycles))
      return false;
    const int c0 = kk * CC;
    const int cn = min(CC, a.C - c0);
    int64_t al[CC], ah[CC];
    uint32_t bytes = 0;
#pragma unroll
    for (int j = 0; j < CC; ++j) {
      if (j >= cn) break;
      const int64_t c = c0 + j;
      const int64_t lo = t0 + __ldg(a.delaysT + c * a.n_dm_pad + i0);
      const int64_t hi = t0 + nt + __ldg(a.delaysT + c * a.n_dm_pad + i0 + BD - 1);
      al[j] = lo & ~(int64_t)(V - 1);
      ah[j] = (hi + V - 1) & ~(int64_t)(V - 1);
      bytes += (uint32_t)((ah[j] - al[j]) * 4) + WD * 16;
    }
    mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
    for (int j = 0; j < CC; ++j) {
      if (j >= cn) break;
      const int64_t c = c0 + j;
      bulk_g2s(sin + (size_t)(s * CC + j) * pitch, in + c * a.in_stride + al[j], (uint32_t)((ah[j] - al[j]) * 4),
               &full[s]);
      bulk_g2s(sdesc + (s * CC + j) * WD, a.regwin_desc + c * n_groups + g0, WD * 16, &full[s]);
    }
    return true;
  };
  int issued = 0;  // meaningful in thread 0 only
  bool prod_failed = false;
  if (tid == 0) {
    for (int kk = 0; kk < min(STAGES, nchunks); ++kk) produce(kk);
    issued = min(STAGES, nchunks);
  }

  // -------------------------------------------------------------- consumers
  const int wd = warp % WD, wt = warp / WD;
  const int lane_t = wt * 32 * SPL + lane * SPL;  // this lane's first sample in the block
  float acc[kRwGroup][SPL];
#pragma unroll
  for (int j = 0; j < kRwGroup; ++j)
#pragma unroll
    for (int q = 0; q < SPL; ++q) acc[j][q] = 0.0f;
  float win[NWIN];
#pragma unroll
  for (int q = 0; q < NWIN; ++q) win[q] = 0.0f;

  bool ok = true;
  for (int k = 0; k < nchunks; ++k) {
    const int s = k % STAGES;
    if (tid == 0 && k >= 1 && issued < nchunks && !prod_failed) {
      if (produce(issued)) {
        ++issued;
      } else {
        prod_failed = true;
        report_error(a.status, kDevWaitTimeout);
        atomicExch(&failed, 1);
      }
    }
    if (!mbar_wait_bounded(&full[s], (uint32_t)((k / STAGES) & 1), kWaitLimitCycles)) {
      if (lane == 0) {
        report_error(a.status, kDevWaitTimeout);
        atomicExch(&failed, 1);
      }
      ok = false;
      break;
    }
    const int c0 = k * CC;
    const int cn = min(CC, a.C - c0);
    for (int j = 0; j < cn; ++j) {
      const int4 dblk = sdesc[(s * CC + j) * WD];      // x = delay(c, i0)
      const int4 dsc = sdesc[(s * CC + j) * WD + wd];  // this warp's group
      // position of (trial i_g, sample t0) in the 16-byte aligned span
      const int r0 = (int)((t0 + dblk.x) & (V - 1)) + (dsc.x - dblk.x) + lane_t;
      const uint32_t saddr = smem_u32(sin + (size_t)(s * CC + j) * pitch) + 4u * (uint32_t)r0;
      RwDispatch<SPL>::load(win, (uint32_t)dsc.w & 0x1fu, saddr);
      const uint32_t lo4 = (uint32_t)dsc.y, hi4 = (uint32_t)dsc.z;
      if constexpr (WEIGHTED) {
        const float wc = __ldg(a.w + c0 + j);
#pragma unroll
        for (int g = 0; g < 4; ++g) RwDispatch<SPL>::fma(acc[g], win, byte_of(lo4, g), wc);
#pragma unroll
        for (int g = 0; g < 4; ++g) RwDispatch<SPL>::fma(acc[4 + g], win, byte_of(hi4, g), wc);
      } else {
#pragma unroll
        for (int g = 0; g < 4; ++g) RwDispatch<SPL>::add(acc[g], win, byte_of(lo4, g));
#pragma unroll
        for (int g = 0; g < 4; ++g) RwDispatch<SPL>::add(acc[4 + g], win, byte_of(hi4, g));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

  // Normally every chunk's copies have landed (each was waited on).  After an
  // expired wait, thread 0 still lets any copy it issued land before leaving.
  if (tid == 0 && (!ok || prod_failed)) {
    for (int kk = max(0, issued - STAGES); kk < issued; ++kk)
      (void)mbar_wait_bounded(&full[kk % STAGES], (uint32_t)((kk / STAGES) & 1), kWaitLimitCycles);
  }
  __syncthreads();
  if (failed) return;
  float* epi = reinterpret_cast<float*>(smem_raw + kRwBarBytes) + (size_t)warp * kRwGroup * 32 * SPL;
#pragma unroll
  for (int j = 0; j < kRwGroup; ++j)
#pragma unroll
    for (int q = 0; q < SPL; ++q) epi[j * 32 * SPL + lane * SPL + q] = acc[j][q];
  __syncwarp();
  float* __restrict__ out = static_cast<float*>(a.out);
  const int tw0 = wt * 32 * SPL;
  const int lim = min(32 * SPL, nt - tw0);
  for (int j = 0; j < kRwGroup; ++j) {
    const int i = i0 + wd * kRwGroup + j;
    if (i >= a.n_dm) break;
    float* orow = out + (int64_t)i * a.out_stride + t0 + tw0;
    for (int u = lane; u < lim; u += 32) orow[u] = epi[j * 32 * SPL + u];
  }
}

// ------------------------------------------------------------------ launch

#define DD_REGWIN_CASES(X) \
  X(4, 2, 15, 8, 4)        \
  X(4, 2, 15, 4, 6)        \
  X(2, 4, 15, 8, 4)        \
  X(4, 1, 15, 8, 4)        \
  X(8, 1, 15, 4, 4)        \
  X(4, 2, 11, 8, 4)        \
  X(2, 2, 15, 8, 3)

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
#define X(WD_, WT_, SPL_, CC_, ST_)                                                                    \
  v.push_back({Kind::RegWin, kRwGroup * WD_, 32 * SPL_ * WT_, CC_, ST_, 32 * WD_ * WT_, SPL_, 0, 0, \
               "regwin_f32_w" #WD_ "x" #WT_ "_s" #SPL_ "_c" #CC_ "_st" #ST_});
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
