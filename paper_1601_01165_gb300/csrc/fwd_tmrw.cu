// TMRW forward kernel (float32): DM-trial reuse through Tensor Memory.
//
// Section 2 observes that nearby DM trials need the same or nearly the same
// input samples, and Section 2.2 exploits it by giving each work group several
// DMs that share loads.  On GB300 one shared-memory load per add (the STAGED
// kernel) caps the sums at a quarter of the FP32 add rate, and a run-time
// offset cannot index registers.  This kernel keeps the reuse but moves the
// run-time offset into an address:
//
//  * a warp owns 4 consecutive DM trials and 32 * SPL samples; lane l owns
//    samples [l*SPL, (l+1)*SPL);
//  * per channel, trial g of the warp needs the lane's samples at offset o_g
//    (0 = o_0 <= o_1 <= o_2 <= o_3) past the first trial's delay; the plan
//    stores the offsets per (channel, 4-trial group) in a 16-byte descriptor;
//  * the lane loads its window of SPL + o_3 samples from the staged span once
//    and stores it into its own row of Tensor Memory (tcgen05.st: TMEM rows
//    are per lane, like registers);
//  * each trial reads its SPL samples back with one tcgen05.ld at column o_g.
//    The offset is the same for the whole warp and part of the TMEM address,
//    so there is no branch and no register indexing.
//
// Software pipeline per warp: the TMEM loads of channel c+1 are in flight
// while the sums of channel c run and the window of channel c+2 is staged
// (two TMEM window buffers, two register buffers), so the TMEM round trip is
// hidden behind useful work.
//
// Staging: each channel's span [t0 + delay(c, i0), t0 + BT + delay(c, i0+BD-1))
// reaches shared memory by 1-D bulk copies, CC channels per stage in a
// STAGES-deep ring with full/empty mbarriers; the producer is lane 0 of warp
// 0 and refills a stage one chunk behind its own progress, so it rarely waits.
// The sums leave through a shared-memory transpose for contiguous stores.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"
#include "ptx.cuh"

namespace dd {

constexpr int kTmBarBytes = 128;
constexpr int kTmSpl = 15;       // samples per lane (odd: lanes' windows start in distinct banks)
constexpr int kTmG = 4;          // DM trials per warp
constexpr uint32_t kTmBuf = 64;  // TMEM columns per window buffer (>= SPL + 31)
constexpr uint32_t kTmCols = 256;  // per block: 2 warps per quadrant x 2 buffers x 64 columns
static_assert(kTmSpl + kRwMaxOff <= 48, "window is stored as 32 + 16 columns");

__host__ __device__ constexpr int tmrw_stage_bytes(int stages, int cc, int wd, int pitch) {
  return kTmBarBytes + stages * cc * pitch * 4 + stages * cc * wd * 16;
}
__host__ __device__ constexpr int tmrw_epi_bytes(int nw) { return kTmBarBytes + nw * kTmG * 32 * kTmSpl * 4; }

__device__ __forceinline__ uint32_t tm_off(uint32_t v, int k) { return (v >> (8 * k)) & 0x1fu; }

template <bool WEIGHTED, int WD, int WT, int CC, int STAGES>
__global__ void __launch_bounds__(32 * WD * WT, 1) fwd_tmrw_f32_kernel(FwdArgs a, int pitch) {
  constexpr int V = 4;
  constexpr int SPL = kTmSpl;
  constexpr int NW = WD * WT;
  constexpr int BD = kTmG * WD;
  constexpr int BT = 32 * SPL * WT;
  static_assert(NW == 8, "two warps per TMEM quadrant");
  static_assert(BT % V == 0, "block start keeps the 16-byte span arithmetic exact");
  static_assert(2 * STAGES * 8 <= kTmBarBytes, "barrier area");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + STAGES;
  float* sin = reinterpret_cast<float*>(smem_raw + kTmBarBytes);
  int4* sdesc = reinterpret_cast<int4*>(smem_raw + kTmBarBytes + (size_t)STAGES * CC * pitch * 4);
  __shared__ uint32_t s_tbase;
  __shared__ int failed;

  const float* __restrict__ in = static_cast<const float*>(a.in);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t t0 = (int64_t)blockIdx.x * BT;
  const int i0 = blockIdx.y * BD;
  const int q0 = i0 / kTmG;  // first 4-trial group of the block
  const int n_quads = a.n_dm_pad / kTmG;
  const int nt = (int)min((int64_t)BT, a.n_out - t0);
  const int C = a.C;
  const int nchunks = (C + CC - 1) / CC;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NW);
    }
    failed = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&s_tbase, kTmCols);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t trow = s_tbase + ((uint32_t)(32 * (warp % 4)) << 16) + 2u * kTmBuf * (uint32_t)(warp / 4);

  // ---------------------------------------------------------------- producer
  auto produce = [&](int kk) -> bool {
    const int s = kk % STAGES;
    if (kk >= STAGES && !mbar_wait_bounded(&empty[s], (uint32_t)(((kk / STAGES) - 1) & 1), kWaitLimitCycles))
      return false;
    const int c0 = kk * CC;
    const int cn = min(CC, C - c0);
    // span of channel c, 16-byte aligned (recomputed rather than kept in
    // registers: this runs inside the consumers' register-heavy loop)
    auto span = [&](int64_t c, int64_t& al, int64_t& ah) {
      const int64_t lo = t0 + __ldg(a.delaysT + c * a.n_dm_pad + i0);
      const int64_t hi = t0 + nt + __ldg(a.delaysT + c * a.n_dm_pad + i0 + BD - 1);
      al = lo & ~(int64_t)(V - 1);
      ah = (hi + V - 1) & ~(int64_t)(V - 1);
    };
    uint32_t bytes = 0;
    for (int j = 0; j < cn; ++j) {
      int64_t al, ah;
      span(c0 + j, al, ah);
      bytes += (uint32_t)((ah - al) * 4) + WD * 16;
    }
    mbar_arrive_expect_tx(&full[s], bytes);
    for (int j = 0; j < cn; ++j) {
      const int64_t c = c0 + j;
      int64_t al, ah;
      span(c, al, ah);
      bulk_g2s(sin + (size_t)(s * CC + j) * pitch, in + c * a.in_stride + al, (uint32_t)((ah - al) * 4), &full[s]);
      bulk_g2s(sdesc + (s * CC + j) * WD, a.quad_desc + c * n_quads + q0, WD * 16, &full[s]);
    }
    return true;
  };
  int issued = 0;
  bool prod_failed = false;
  if (tid == 0) {
    for (int kk = 0; kk < min(STAGES, nchunks); ++kk) produce(kk);
    issued = min(STAGES, nchunks);
  }

  // ---------------------------------------------------------------- consumer
  const int wd = warp % WD, wt = warp / WD;
  const int lane_t = wt * 32 * SPL + lane * SPL;
  int waited = 0;      // chunks whose full barrier this warp has passed
  bool ok = true;

  // Make chunk c / CC visible to this warp (warp-uniform result).
  auto ensure = [&](int c) -> bool {
    const int kk = c / CC;
    while (waited <= kk) {
      const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&full[waited % STAGES],
                                                                 (uint32_t)((waited / STAGES) & 1), kWaitLimitCycles));
      if (!got) return false;
      ++waited;
    }
    return true;
  };
  // After the last read of chunk c / CC: release its stage; lane 0 of warp 0
  // then refills the stage freed one chunk earlier.
  auto release = [&](int c) {
    if (c % CC != CC - 1 && c != C - 1) return;
    const int kk = c / CC;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[kk % STAGES]);
    if (tid == 0 && kk >= 1 && !prod_failed && issued < nchunks) {
      if (produce(issued)) {
        ++issued;
      } else {
        prod_failed = true;
        report_error(a.status, kDevWaitTimeout);
        atomicExch(&failed, 1);
      }
    }
    __syncwarp();
  };
  // Window of channel c -> TMEM buffer b; returns the warp's descriptor for c.
  auto window = [&](int c, uint32_t b) -> int4 {
    const int s = (c / CC) % STAGES, j = c % CC;
    const int4 dblk = sdesc[(s * CC + j) * WD];
    const int4 dsc = sdesc[(s * CC + j) * WD + wd];
    const int r0 = (int)((t0 + dblk.x) & (V - 1)) + (dsc.x - dblk.x) + lane_t;
    const float* row = sin + (size_t)(s * CC + j) * pitch + r0;
    const int nwin = SPL + (dsc.z & 0x1f);
    float win[32];
#pragma unroll
    for (int q = 0; q < 16; ++q) win[q] = row[q];
#pragma unroll
    for (int q = 16; q < 32; ++q) win[q] = 0.0f;
    if (nwin > 16) {
#pragma unroll
      for (int q = 16; q < 24; ++q) win[q] = row[q];
      if (nwin > 24) {
#pragma unroll
        for (int q = 24; q < 32; ++q) win[q] = row[q];
      }
    }
    tmem_st32(trow + kTmBuf * b, win);
    if (nwin > 32) {
      float w2[16];
#pragma unroll
      for (int q = 0; q < 8; ++q) w2[q] = row[32 + q];
#pragma unroll
      for (int q = 8; q < 16; ++q) w2[q] = 0.0f;
      if (nwin > 40) {
#pragma unroll
        for (int q = 8; q < 16; ++q) w2[q] = row[32 + q];
      }
      tmem_st16(trow + kTmBuf * b + 32, w2);
    }
    return dsc;
  };
  auto load = [&](const int4& dsc, uint32_t b, float (&v)[kTmG][16]) {
    const uint32_t tb = trow + kTmBuf * b, offs = (uint32_t)dsc.y;
#pragma unroll
    for (int g = 0; g < kTmG; ++g) tmem_ld16(tb + tm_off(offs, g), v[g]);
  };

  float acc[kTmG][SPL];
#pragma unroll
  for (int g = 0; g < kTmG; ++g)
#pragma unroll
    for (int q = 0; q < SPL; ++q) acc[g][q] = 0.0f;
  float vA[kTmG][16], vB[kTmG][16];
  int4 dX = make_int4(0, 0, 0, 0), dY = make_int4(0, 0, 0, 0);

  // One pipeline step: issue the loads of channel c+1 (descriptor dn1, its
  // window already stored) into `nxt`; sum channel c from `cur`; then stage
  // the window of channel c+2 into the TMEM buffer channel c used (its
  // registers reuse `cur`'s), keeping its descriptor in dn2.
  auto step = [&](int c, float (&cur)[kTmG][16], float (&nxt)[kTmG][16], const int4& dn1, int4& dn2) {
    tmem_wait_st();
    if (c + 1 < C) load(dn1, (uint32_t)((c + 1) & 1), nxt);
    float wc = 1.0f;
    if constexpr (WEIGHTED) wc = __ldg(a.w + c);
#pragma unroll
    for (int g = 0; g < kTmG; ++g)
#pragma unroll
      for (int q = 0; q < SPL; ++q) {
        if constexpr (WEIGHTED) {
          acc[g][q] = fmaf(wc, cur[g][q], acc[g][q]);
        } else {
          acc[g][q] += cur[g][q];
        }
      }
    if (c + 2 < C) {
      if (ensure(c + 2)) {
        dn2 = window(c + 2, (uint32_t)(c & 1));
        release(c + 2);
      } else {
        ok = false;
      }
    }
    tmem_wait_ld();
  };

  // prologue: windows of channels 0 and 1, loads of channel 0
  if (ensure(0)) {
    const int4 d0 = window(0, 0);
    release(0);
    if (C > 1) {
      if (ensure(1)) {
        dX = window(1, 1);
        release(1);
      } else {
        ok = false;
      }
    }
    tmem_wait_st();
    load(d0, 0, vA);
    tmem_wait_ld();
  } else {
    ok = false;
  }
  for (int c = 0; ok && c < C; c += 2) {
    step(c, vA, vB, dX, dY);
    if (!ok || c + 1 >= C) break;
    step(c + 1, vB, vA, dY, dX);
  }
  tmem_wait_st();
  tmem_wait_ld();
  if (!ok && lane == 0) {
    report_error(a.status, kDevWaitTimeout);
    atomicExch(&failed, 1);
  }

  if (tid == 0 && (!ok || prod_failed)) {
    for (int kk = max(0, issued - STAGES); kk < issued; ++kk)
      (void)mbar_wait_bounded(&full[kk % STAGES], (uint32_t)((kk / STAGES) & 1), kWaitLimitCycles);
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(s_tbase, kTmCols);
  if (failed) return;

  float* epi = reinterpret_cast<float*>(smem_raw + kTmBarBytes) + (size_t)warp * kTmG * 32 * SPL;
#pragma unroll
  for (int g = 0; g < kTmG; ++g)
#pragma unroll
    for (int q = 0; q < SPL; ++q) epi[g * 32 * SPL + lane * SPL + q] = acc[g][q];
  __syncwarp();
  float* __restrict__ out = static_cast<float*>(a.out);
  const int tw0 = wt * 32 * SPL;
  const int lim = min(32 * SPL, nt - tw0);
  for (int g = 0; g < kTmG; ++g) {
    const int i = i0 + wd * kTmG + g;
    if (i >= a.n_dm) break;
    float* orow = out + (int64_t)i * a.out_stride + t0 + tw0;
    for (int u = lane; u < lim; u += 32) orow[u] = epi[g * 32 * SPL + u];
  }
}

#define DD_TMRW_CASES(X) \
  X(8, 1, 8, 4)          \
  X(8, 1, 4, 6)          \
  X(4, 2, 8, 4)          \
  X(4, 2, 4, 6)          \
  X(2, 4, 8, 4)

template <bool W, int WD, int WT, int CC, int STAGES>
static cudaError_t launch_tm_t(const TileConfig& cfg, const FwdArgs& a, cudaStream_t s) {
  auto kern = fwd_tmrw_f32_kernel<W, WD, WT, CC, STAGES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cfg.smem);
  if (e != cudaSuccess) return e;
  constexpr int BD = kTmG * WD, BT = 32 * kTmSpl * WT;
  dim3 grid((unsigned)((a.n_out + BT - 1) / BT), (unsigned)((a.n_dm + BD - 1) / BD));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  kern<<<grid, 32 * WD * WT, cfg.smem, s>>>(a, cfg.pitch);
  return cudaGetLastError();
}

cudaError_t launch_tmrw(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s) {
  if (dtype != DD_F32_F32) return cudaErrorInvalidConfiguration;
  const bool w = a.w != nullptr;
#define X(WD_, WT_, CC_, ST_)                                                                          \
  if (cfg.bd == kTmG * WD_ && cfg.bt == 32 * kTmSpl * WT_ && cfg.cc == CC_ && cfg.stages == ST_)     \
    return w ? launch_tm_t<true, WD_, WT_, CC_, ST_>(cfg, a, s) : launch_tm_t<false, WD_, WT_, CC_, ST_>(cfg, a, s);
  DD_TMRW_CASES(X)
#undef X
  return cudaErrorInvalidConfiguration;
}

std::vector<TileConfig> tmrw_menu(dd_dtype dtype) {
  std::vector<TileConfig> v;
  if (dtype != DD_F32_F32) return v;
#define X(WD_, WT_, CC_, ST_)                                                                      \
  v.push_back({Kind::TmRw, kTmG * WD_, 32 * kTmSpl * WT_, CC_, ST_, 32 * WD_ * WT_, kTmSpl, 0, 0, \
               "tmrw_f32_w" #WD_ "x" #WT_ "_c" #CC_ "_st" #ST_});
  DD_TMRW_CASES(X)
#undef X
  return v;
}

int tmrw_smem_for(const TileConfig& cfg, int pitch) {
  const int wd = cfg.bd / kTmG;
  const int a = tmrw_stage_bytes(cfg.stages, cfg.cc, wd, pitch);
  const int b = tmrw_epi_bytes(cfg.threads / 32);
  return a > b ? a : b;
}

}  // namespace dd
