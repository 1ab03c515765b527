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

#include <algorithm>
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
// slices.
constexpr int kStBarBytes = 128;
template <typename Tin>
__host__ __device__ constexpr int staged_smem_bytes(int stages, int cc, int bd, int pitch) {
  return kStBarBytes + stages * cc * pitch * (int)sizeof(Tin) + stages * cc * bd * 4;
}

// The stage barriers: full[s] completes when stage s's copies have landed
// (one arrival per copying warp with the bytes that warp copies, then the
// bytes); empty[s] when every warp of the block has finished reading it (one
// arrival per warp).  Warps synchronise only through these, never block-wide
// inside the channel loop.
template <int STAGES>
struct StageBars {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
};

template <int STAGES>
__device__ __forceinline__ StageBars<STAGES>& init_stage_bars(unsigned char* smem_raw, int warps, int copiers) {
  static_assert(sizeof(StageBars<STAGES>) <= kStBarBytes, "barrier area");
  StageBars<STAGES>& B = *reinterpret_cast<StageBars<STAGES>*>(smem_raw);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&B.full[s], (uint32_t)copiers);
      mbar_init(&B.empty[s], (uint32_t)warps);
    }
    fence_mbar_init();
  }
  __syncthreads();
  return B;
}

// Fresh barriers for a persistent block's next tile.  Called by every thread
// once the block is past its tile: every copy has landed (the copiers drained
// them) and no thread waits on or arrives at the old barriers any more.
template <int STAGES>
__device__ __forceinline__ void reset_stage_bars(StageBars<STAGES>& B, int warps, int copiers) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_inval(&B.full[s]);
      mbar_inval(&B.empty[s]);
      mbar_init(&B.full[s], (uint32_t)copiers);
      mbar_init(&B.empty[s], (uint32_t)warps);
    }
    fence_mbar_init();
  }
  __syncthreads();
}

// The warps of a STAGED or U8PK block copy their own input: chunk k
// (channels [k CC, k CC + CC)) goes to stage k % STAGES, one lane per slot j
// (the span of channel k CC + j and its BD delays).  With SPREAD every warp
// copies part of each chunk (lane l of warp w takes slot w + NW l), so no warp
// carries all the copies; without it warp 0 copies everything (lane l takes
// slot l).  U8PK, which has few shared loads per add, runs fastest spread;
// STAGED, bound by shared-memory bandwidth, with warp 0 alone.  A lane reads
// its channel's first and last trial delays one chunk before it stages that
// chunk (stage_fetch), so the delay-table latency stays off the warp's path.
template <int BD, int CC>
__device__ __forceinline__ void stage_fetch(const FwdArgs& a, int i0, int k, int slot, int32_t& dlo, int32_t& dhi) {
  const int c = k * CC + slot;
  if (slot < CC && c < a.C) {
    const int32_t* col = a.delaysT + (int64_t)c * a.n_dm_pad + i0;
    dlo = __ldg(col);
    dhi = __ldg(col + BD - 1);
  }
}

// All lanes of a warp: stage the warp's slots of chunk k into stage s
// (barrier `bar`) from the delays stage_fetch read.  Each span covers samples
// [t0 + dlo, t0 + nt + dhi) of its channel row, widened to 16-byte boundaries.
template <typename Tin, int BD, int CC>
__device__ __forceinline__ void stage_issue(const FwdArgs& a, int pitch, int64_t t0, int nt, int i0, int k, int s,
                                            int slot, int lane, int32_t dlo, int32_t dhi, uint64_t* bar, Tin* sin,
                                            int32_t* sdel) {
  constexpr int V = 16 / (int)sizeof(Tin);
  const int c = k * CC + slot;
  const bool mine = slot < CC && c < a.C;
  int64_t al = 0, ah = 0;
  if (mine) {
    al = (t0 + dlo) & ~(int64_t)(V - 1);
    ah = (t0 + nt + dhi + V - 1) & ~(int64_t)(V - 1);
    // the span fits its shared-memory row and its input row
    if (!DD_INDEX_OK(a.status, al >= 0 && ah - al <= pitch && ah <= a.in_stride)) al = 0, ah = V;
  }
  const uint32_t bytes = mine ? (uint32_t)((ah - al) * (int64_t)sizeof(Tin)) + BD * 4 : 0u;
  const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
  if (lane == 0) mbar_arrive_expect_tx(bar, total);
  __syncwarp();
  if (mine) {
    bulk_g2s(sin + (size_t)(s * CC + slot) * pitch, static_cast<const Tin*>(a.in) + (int64_t)c * a.in_stride + al,
             (uint32_t)((ah - al) * (int64_t)sizeof(Tin)), bar);
    bulk_g2s(sdel + (s * CC + slot) * BD, a.delaysT + (int64_t)c * a.n_dm_pad + i0, BD * 4, bar);
  }
}

// A copying warp's side of the pipeline: `kn` is the next chunk it stages
// and (dlo, dhi) its lanes' delays for it.  Every tile starts on fresh
// barriers (a persistent block resets them between tiles).
template <typename Tin, int BD, int CC, int STAGES, int NW, bool SPREAD>
struct Stager {
  static_assert(STAGES >= 2, "chunk k + 1 is staged while chunk k is read");
  static_assert(CC <= (SPREAD ? 32 * NW : 32), "one lane per slot of a chunk");
  static constexpr int kCopiers = SPREAD ? NW : 1;  // warps that copy
  const FwdArgs& a;
  int pitch;
  int64_t t0;
  int nt, i0, nchunks, warp, lane;
  StageBars<STAGES>& B;
  Tin* sin;
  int32_t* sdel;
  int kn = 0;
  int32_t dlo = 0, dhi = 0;

  // does this warp copy, and which chunk slot does this lane copy
  __device__ __forceinline__ bool copies() const { return SPREAD || warp == 0; }
  __device__ __forceinline__ int slot() const { return SPREAD ? warp + NW * lane : lane; }

  // Stage the first min(STAGES, nchunks) chunks (their stages start free),
  // reading all their delays at once.
  __device__ __forceinline__ void prologue() {
    int32_t plo[STAGES], phi[STAGES];
#pragma unroll
    for (int j = 0; j < STAGES; ++j) {
      plo[j] = phi[j] = 0;
      stage_fetch<BD, CC>(a, i0, j, slot(), plo[j], phi[j]);
    }
#pragma unroll
    for (int j = 0; j < STAGES; ++j)
      if (j < nchunks)
        stage_issue<Tin, BD, CC>(a, pitch, t0, nt, i0, j, j, slot(), lane, plo[j], phi[j], &B.full[j], sin, sdel);
    kn = min(STAGES, nchunks);
    stage_fetch<BD, CC>(a, i0, STAGES, slot(), dlo, dhi);
  }

  // Called by a copying warp before it consumes chunk k: stage, in order, its part of every chunk
  // up to k + STAGES - 1 whose stage every warp has released (chunk kn's stage
  // is free once chunk kn - STAGES is released).  Chunks k and k + 1 must be
  // staged by now, so their stages are waited for (bounded; this keeps at
  // least one chunk of copies ahead of the sums); later ones are only staged
  // if already free.  False on a timeout.
  __device__ __forceinline__ bool ahead(int k) {
    const int upto = min(nchunks, k + STAGES);
    while (kn < upto) {
      const int s = kn % STAGES;
      const uint32_t par = (uint32_t)(((kn - STAGES) / STAGES) & 1);
      if (!__any_sync(0xffffffffu, mbar_test_wait(&B.empty[s], par))) {
        if (kn > k + 1) break;  // try again at the next chunk
        if (!__any_sync(0xffffffffu, mbar_wait_bounded(&B.empty[s], par, kWaitLimitCycles))) return false;
      }
      stage_issue<Tin, BD, CC>(a, pitch, t0, nt, i0, kn, s, slot(), lane, dlo, dhi, &B.full[s], sin, sdel);
      stage_fetch<BD, CC>(a, i0, kn + 1, slot(), dlo, dhi);
      ++kn;
    }
    return true;
  }

  // Before the block reuses the stages or leaves: no copy may still be in
  // flight (after a timeout some staged chunks were never consumed).
  __device__ __forceinline__ void drain() {
    if (lane == 0)
      for (int kk = max(0, kn - STAGES); kk < kn; ++kk)
        (void)mbar_wait_bounded(&B.full[kk % STAGES], (uint32_t)((kk / STAGES) & 1), kWaitLimitCycles);
    __syncwarp();
  }
};

// Every warp: wait for chunk k's stage to be full (bounded, warp-uniform).
template <int STAGES>
__device__ __forceinline__ bool stage_wait_full(StageBars<STAGES>& B, int k) {
  return __all_sync(0xffffffffu, mbar_wait_bounded(&B.full[k % STAGES], (uint32_t)((k / STAGES) & 1), kWaitLimitCycles));
}

// Every warp, after reading chunk k's stage: release it.
template <int STAGES>
__device__ __forceinline__ void stage_release(StageBars<STAGES>& B, int k, int lane) {
  __syncwarp();
  if (lane == 0) mbar_arrive(&B.empty[k % STAGES]);
}

// One tile: DM trials [i0, i0 + BD) x samples [t0, t0 + BT), on fresh stage
// barriers.  False after a timeout (also reported in the status word).
template <typename Tin, bool WEIGHTED, int BD, int BT, int CC, int STAGES>
__device__ __forceinline__ bool staged_tile(const FwdArgs& a, int pitch, int64_t t0, int i0,
                                            StageBars<STAGES>& B, unsigned char* smem_raw) {
  using Tacc = typename AccOf<Tin>::type;
  constexpr int V = 16 / (int)sizeof(Tin);  // elements per 16 bytes
  constexpr int NW = 8;
  constexpr int DPW = BD / NW;
  constexpr int SPL = BT / 32;
  static_assert(BD % NW == 0 && BT % 64 == 0 && BD % 4 == 0, "tile shape (an even number of samples per lane)");
  // a block's delay slice [i0, i0 + BD) must stay inside the padded row
  static_assert(kDmPad % BD == 0, "BD must divide the trial padding");
  using Pipe = Stager<Tin, BD, CC, STAGES, NW, false>;
  Tin* sin = reinterpret_cast<Tin*>(smem_raw + kStBarBytes);
  int32_t* sdel = reinterpret_cast<int32_t*>(smem_raw + kStBarBytes + (size_t)STAGES * CC * pitch * sizeof(Tin));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = (int)min((int64_t)BT, a.n_out - t0);
  const int nchunks = (a.C + CC - 1) / CC;

  Pipe st{a, pitch, t0, nt, i0, nchunks, warp, lane, B, sin, sdel};
  bool ok = true;
  if (st.copies()) st.prologue();

  Tacc acc[DPW][SPL];
#pragma unroll
  for (int m = 0; m < DPW; ++m)
#pragma unroll
    for (int q = 0; q < SPL; ++q) acc[m][q] = 0;

  for (int k = 0; k < nchunks && ok; ++k) {
    if (st.copies() && !st.ahead(k)) {
      ok = false;
      break;
    }
    if (!stage_wait_full(B, k)) {
      ok = false;
      break;
    }
    const int s = k % STAGES;
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
        if constexpr (sizeof(Tin) == 4) {
          // float: packed pairs of adds (same results, half the add instructions)
#pragma unroll
          for (int q = 0; q < SPL; q += 2) {
            if constexpr (WEIGHTED) {
              fma2_rn(acc[m][q], acc[m][q + 1], wc, row[off + 32 * q], row[off + 32 * q + 32]);
            } else {
              add2_rn(acc[m][q], acc[m][q + 1], row[off + 32 * q], row[off + 32 * q + 32]);
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < SPL; ++q) acc[m][q] += (Tacc)row[off + 32 * q];
        }
      }
    }
    stage_release(B, k, lane);
  }
  if (st.copies()) st.drain();
  if (!ok) {
    if (lane == 0) report_error(a.status, kDevWaitTimeout);
    return false;
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
  return true;
}

template <typename Tin, bool WEIGHTED, int BD, int BT, int CC, int STAGES>
__global__ void __launch_bounds__(256) fwd_staged_kernel(FwdArgs a, int pitch) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  StageBars<STAGES>& B = init_stage_bars<STAGES>(smem_raw, 8, Stager<Tin, BD, CC, STAGES, 8, false>::kCopiers);
  (void)staged_tile<Tin, WEIGHTED, BD, BT, CC, STAGES>(a, pitch, (int64_t)blockIdx.x * BT, blockIdx.y * BD, B,
                                                        smem_raw);
}

// Persistent form for batches: the block takes tiles of many beams from the
// work list until it is exhausted (see BatchWork), each tile exactly as a
// block of the plain kernel runs it, on stage barriers reset in between.
template <typename Tin, bool WEIGHTED, int BD, int BT, int CC, int STAGES>
__global__ void __launch_bounds__(256) fwd_staged_persistent(const __grid_constant__ BatchWork w) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int kCopiers = Stager<Tin, BD, CC, STAGES, 8, false>::kCopiers;
  StageBars<STAGES>& B = init_stage_bars<STAGES>(smem_raw, 8, kCopiers);
  __shared__ int item_s;
  __shared__ BatchBeam beam_s;  // the tile's arguments, at fixed shared addresses
  while (true) {
    WorkItem it;
    if (!next_item(w, item_s, it)) break;
    copy_beam(w, it.beam, beam_s);
    const bool ok = staged_tile<Tin, WEIGHTED, BD, BT, CC, STAGES>(beam_s.a, beam_s.pitch, (int64_t)it.x * BT,
                                                                    it.y * BD, B, smem_raw);
    if (__syncthreads_or(!ok)) break;
    reset_stage_bars<STAGES>(B, 8, kCopiers);
  }
}

// ------------------------------------------------------------------- U8PK
// uint8 -> int32 with packed accumulation.  The block stages byte spans
// exactly like STAGED.  A warp owns DPW DM trials x 32 lanes x 28 samples (7
// words; odd, so the lanes' word loads hit distinct banks).  Per channel and
// trial a lane loads 8 words covering its 28 samples at the trial's delay and
// aligns them with one byte permute whose selector is the same for the whole
// warp (the delay modulo 4).  For each aligned word x = s0 + 2^8 s1 + 2^16 s2
// + 2^24 s3 it keeps two sums: A, the words themselves modulo 2^32, and B, the
// odd samples s1, s3 as two 16-bit lanes.  Over at most 256 channels every
// per-sample sum S_k stays below 2^16 (256 * 255 < 65536), so B holds S1 and
// S3 exactly and A - 2^8 S1 - 2^24 S3 = S0 + 2^16 S2 (mod 2^32) gives S0 and
// S2; every 256 channels the four sums are added into int32 totals and A, B
// cleared, so the result is the exact integer sum.  The sums are formed with
// integer multiply-adds by a run-time 1 so that they issue to the FMA pipe,
// leaving the ALU pipe to the byte permutes (two per word and channel).
template <int WD, int WT, int DPW>
struct U8PkShape {
  static constexpr int KW = 7;        // words per lane
  static constexpr int SPL = 4 * KW;  // samples per lane
  static constexpr int BD = WD * DPW;
  static constexpr int BT = 32 * SPL * WT;
};

// One tile: DM trials [i0, i0 + BD) x samples [t0, t0 + BT), on fresh stage
// barriers.  False after a timeout (also reported).
template <int WD, int WT, int DPW, int CC, int STAGES>
__device__ __forceinline__ bool u8pk_tile(const FwdArgs& a, int pitch, int64_t t0, int i0,
                                          StageBars<STAGES>& B, unsigned char* smem_raw) {
  constexpr int V = 16;
  constexpr int NW = WD * WT;
  constexpr int KW = U8PkShape<WD, WT, DPW>::KW;
  constexpr int SPL = U8PkShape<WD, WT, DPW>::SPL;
  constexpr int BD = U8PkShape<WD, WT, DPW>::BD;
  constexpr int BT = U8PkShape<WD, WT, DPW>::BT;
  static_assert(BD % 4 == 0 && BT % 16 == 0, "tile shape");
  static_assert(kDmPad % BD == 0, "BD must divide the trial padding");
  using Pipe = Stager<uint8_t, BD, CC, STAGES, NW, true>;
  uint8_t* sin = smem_raw + kStBarBytes;
  int32_t* sdel = reinterpret_cast<int32_t*>(smem_raw + kStBarBytes + (size_t)STAGES * CC * pitch);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wd = warp % WD, wt = warp / WD;
  const int nt = (int)min((int64_t)BT, a.n_out - t0);
  const int nchunks = (a.C + CC - 1) / CC;

  Pipe st{a, pitch, t0, nt, i0, nchunks, warp, lane, B, sin, sdel};
  bool ok = true;
  if (st.copies()) st.prologue();

  uint32_t ra[DPW][KW], rb[DPW][KW];  // A and B of each word (see above)
#pragma unroll
  for (int m = 0; m < DPW; ++m)
#pragma unroll
    for (int w = 0; w < KW; ++w) ra[m][w] = rb[m][w] = 0u;
  const int lane_off = wt * 32 * SPL + lane * SPL;  // this lane's first sample in the tile
  // Flush: decode the exact sums since the last flush and add them to the
  // int32 totals, then clear A and B.  With up to two trials per warp the
  // totals stay in registers and leave through a shared-memory transpose at
  // the end; with four there is no room, so each flush adds them straight to
  // the lane's own output samples (the first flush stores them; each lane
  // owns SPL consecutive samples of its trials, so no other thread touches
  // them; 16-byte accesses where the row allows).
  constexpr bool kOutTotals = DPW >= 4;
  int32_t tot[kOutTotals ? 1 : DPW][kOutTotals ? 1 : SPL];
  if constexpr (!kOutTotals) {
#pragma unroll
    for (int m = 0; m < DPW; ++m)
#pragma unroll
      for (int q = 0; q < SPL; ++q) tot[m][q] = 0;
  }
  int32_t* __restrict__ out = static_cast<int32_t*>(a.out);
  const bool vec = (reinterpret_cast<uintptr_t>(a.out) % 16 == 0) && (a.out_stride % 4 == 0);
  const int64_t tl = t0 + lane_off;
  const int nl = (int)max((int64_t)0, min((int64_t)SPL, a.n_out - tl));  // this lane's samples inside the output
  bool first = true;
  auto flush = [&]() {
    if constexpr (!kOutTotals) {
#pragma unroll
      for (int m = 0; m < DPW; ++m)
#pragma unroll
        for (int w = 0; w < KW; ++w) {
          const uint32_t s1 = rb[m][w] & 0xffffu, s3 = rb[m][w] >> 16;
          const uint32_t s02 = ra[m][w] - (s1 << 8) - (s3 << 24);  // S0 + 2^16 S2
          tot[m][4 * w + 0] += (int32_t)(s02 & 0xffffu);
          tot[m][4 * w + 1] += (int32_t)s1;
          tot[m][4 * w + 2] += (int32_t)(s02 >> 16);
          tot[m][4 * w + 3] += (int32_t)s3;
          ra[m][w] = rb[m][w] = 0u;
        }
    } else {
#pragma unroll
      for (int m = 0; m < DPW; ++m) {
        const int i = i0 + wd * DPW + m;
        int32_t* o = out + (int64_t)min(i, a.n_dm - 1) * a.out_stride + tl;
#pragma unroll
        for (int w = 0; w < KW; ++w) {
          const uint32_t s1 = rb[m][w] & 0xffffu, s3 = rb[m][w] >> 16;
          const uint32_t s02 = ra[m][w] - (s1 << 8) - (s3 << 24);  // S0 + 2^16 S2
          int4 v = make_int4((int32_t)(s02 & 0xffffu), (int32_t)s1, (int32_t)(s02 >> 16), (int32_t)s3);
          ra[m][w] = rb[m][w] = 0u;
          if (i >= a.n_dm) continue;
          if (vec && 4 * w + 3 < nl) {
            int4* p4 = reinterpret_cast<int4*>(o + 4 * w);
            if (!first) {
              const int4 u = *p4;
              v.x += u.x, v.y += u.y, v.z += u.z, v.w += u.w;
            }
            *p4 = v;
          } else {  // row end or unaligned rows: one sample at a time
            int32_t* e = o + 4 * w;
            const int k = nl - 4 * w;
            if (k > 0) e[0] = first ? v.x : e[0] + v.x;
            if (k > 1) e[1] = first ? v.y : e[1] + v.y;
            if (k > 2) e[2] = first ? v.z : e[2] + v.z;
            if (k > 3) e[3] = first ? v.w : e[3] + v.w;
          }
        }
      }
    }
    first = false;
  };
  // x + y * one with one == 1 at run time: an integer multiply-add (FMA pipe)
  const uint32_t one = a.C > 0 ? 1u : 0u;
  auto madd = [](uint32_t x, uint32_t y, uint32_t m) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(y), "r"(m), "r"(x));
    return d;
  };
  // The 4 bytes starting at byte (sel mod 4) of the 8 bytes lo, hi (lo first).
  auto f4e = [](uint32_t lo, uint32_t hi, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32.f4e %0, %1, %2, %3;" : "=r"(d) : "r"(lo), "r"(hi), "r"(sel));
    return d;
  };
  // Channel row j of stage s: the row and the offset `cj` such that trial
  // slot i's samples for this lane start at byte cj + dl[i] of the row (the
  // row starts at t0 + dl[0] rounded down to 16 bytes; t0 is a multiple of 16).
  auto channel = [&](int s, int j, const uint8_t*& row, const int32_t*& dl, int& cj) {
    row = sin + (size_t)(s * CC + j) * pitch;
    dl = sdel + (s * CC + j) * BD;
    const int d0 = dl[0];
    cj = (int)(((uint32_t)t0 + (uint32_t)d0) & (uint32_t)(V - 1)) - d0 + lane_off;
  };
  // aligned words of trial slot m of a channel row -> x[KW]
  auto aligned = [&](const uint8_t* row, const int32_t* dl, int cj, int m, uint32_t (&x)[KW]) {
    const int off = cj + dl[wd * DPW + m];
    const uint32_t* wp = reinterpret_cast<const uint32_t*>(row + (off & ~3));
    uint32_t wv[KW + 1];
    // the KW + 1 words stay inside the channel's shared-memory row
    if (!DD_INDEX_OK(a.status, off >= 0 && (off >> 2) + KW + 1 <= pitch / 4)) wp = reinterpret_cast<const uint32_t*>(row);
#pragma unroll
    for (int w = 0; w <= KW; ++w) wv[w] = wp[w];
#pragma unroll
    for (int w = 0; w < KW; ++w) x[w] = f4e(wv[w], wv[w + 1], (uint32_t)off);
  };

  int since_flush = 0;
  for (int k = 0; k < nchunks && ok; ++k) {
    if (st.copies() && !st.ahead(k)) {
      ok = false;
      break;
    }
    if (!stage_wait_full(B, k)) {
      ok = false;
      break;
    }
    const int s = k % STAGES;
    const int cn = min(CC, a.C - k * CC);
    int j = 0;
    for (; j + 1 < cn; j += 2) {
      if (since_flush >= 255) {  // the next two channels would pass 256
        flush();
        since_flush = 0;
      }
      const uint8_t *row0, *row1;
      const int32_t *dl0, *dl1;
      int c0j, c1j;
      channel(s, j, row0, dl0, c0j);
      channel(s, j + 1, row1, dl1, c1j);
#pragma unroll
      for (int m = 0; m < DPW; ++m) {
        uint32_t x0[KW], x1[KW];
        aligned(row0, dl0, c0j, m, x0);
        aligned(row1, dl1, c1j, m, x1);
#pragma unroll
        for (int w = 0; w < KW; ++w) {
          ra[m][w] = madd(madd(ra[m][w], x0[w], one), x1[w], one);
          rb[m][w] = madd(madd(rb[m][w], __byte_perm(x0[w], 0u, 0x4341u), one), __byte_perm(x1[w], 0u, 0x4341u), one);
        }
      }
      since_flush += 2;
    }
    if (j < cn) {
      if (since_flush >= 256) {
        flush();
        since_flush = 0;
      }
      const uint8_t* row0;
      const int32_t* dl0;
      int c0j;
      channel(s, j, row0, dl0, c0j);
#pragma unroll
      for (int m = 0; m < DPW; ++m) {
        uint32_t x0[KW];
        aligned(row0, dl0, c0j, m, x0);
#pragma unroll
        for (int w = 0; w < KW; ++w) {
          ra[m][w] = madd(ra[m][w], x0[w], one);
          rb[m][w] = madd(rb[m][w], __byte_perm(x0[w], 0u, 0x4341u), one);
        }
      }
      since_flush += 1;
    }
    stage_release(B, k, lane);
  }
  if (ok) flush();
  if (st.copies()) st.drain();
  if (!ok && lane == 0) report_error(a.status, kDevWaitTimeout);
  if constexpr (!kOutTotals) {
    // transpose through shared memory (every warp is past the channel loop
    // and no copy is in flight, so the stage area is free); the block agrees
    // on the outcome first, so every warp meets the barriers below or none
    if (!__syncthreads_and(ok)) return false;
    int32_t* epi = reinterpret_cast<int32_t*>(smem_raw + kStBarBytes) + (size_t)warp * DPW * 32 * SPL;
#pragma unroll
    for (int m = 0; m < DPW; ++m)
#pragma unroll
      for (int q = 0; q < SPL; ++q) epi[m * 32 * SPL + lane * SPL + q] = tot[m][q];
    __syncwarp();
    const int tw0 = wt * 32 * SPL;
    const int lim = min(32 * SPL, nt - tw0);
    for (int m = 0; m < DPW; ++m) {
      const int i = i0 + wd * DPW + m;
      if (i >= a.n_dm) break;
      int32_t* orow = out + (int64_t)i * a.out_stride + t0 + tw0;
      for (int u = lane; u < lim; u += 32) orow[u] = epi[m * 32 * SPL + u];
    }
    // the next tile of a persistent block stages into this area again
    __syncthreads();
  }
  return ok;
}

template <int WD, int WT, int DPW, int CC, int STAGES>
__global__ void __launch_bounds__(32 * WD * WT) fwd_u8pk_kernel(FwdArgs a, int pitch) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  using Sh = U8PkShape<WD, WT, DPW>;
  StageBars<STAGES>& B =
      init_stage_bars<STAGES>(smem_raw, WD * WT, Stager<uint8_t, Sh::BD, CC, STAGES, WD * WT, true>::kCopiers);
  (void)u8pk_tile<WD, WT, DPW, CC, STAGES>(a, pitch, (int64_t)blockIdx.x * Sh::BT, blockIdx.y * Sh::BD, B, smem_raw);
}

// Persistent form for batches (see fwd_staged_persistent).
template <int WD, int WT, int DPW, int CC, int STAGES>
__global__ void __launch_bounds__(32 * WD * WT) fwd_u8pk_persistent(const __grid_constant__ BatchWork w) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  using Sh = U8PkShape<WD, WT, DPW>;
  constexpr int kCopiers = Stager<uint8_t, Sh::BD, CC, STAGES, WD * WT, true>::kCopiers;
  StageBars<STAGES>& B = init_stage_bars<STAGES>(smem_raw, WD * WT, kCopiers);
  __shared__ int item_s;
  while (true) {
    WorkItem it;
    if (!next_item(w, item_s, it)) break;
    const BatchBeam& bm = w.beams[it.beam];  // kernel parameters
    const bool ok =
        u8pk_tile<WD, WT, DPW, CC, STAGES>(bm.a, bm.pitch, (int64_t)it.x * Sh::BT, it.y * Sh::BD, B, smem_raw);
    if (__syncthreads_or(!ok)) break;
    reset_stage_bars<STAGES>(B, WD * WT, kCopiers);
  }
}

// Stages, and with up to two trials per warp room for the final transpose.
__host__ __device__ constexpr int u8pk_smem_bytes(int stages, int cc, int bd, int pitch, int nw, int dpw) {
  return (dpw >= 4 || stages * cc * pitch + stages * cc * bd * 4 > nw * dpw * 32 * 28 * 4)
             ? kStBarBytes + stages * cc * pitch + stages * cc * bd * 4
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
  X(64, 256, 4, 3)           \
  X(32, 512, 2, 4)           \
  X(32, 512, 8, 2)           \
  X(32, 384, 4, 3)

#define DD_U8PK_CASES(X) \
  X(8, 1, 2, 16, 4)      \
  X(4, 2, 2, 16, 4)      \
  X(8, 1, 4, 16, 3)      \
  X(4, 1, 2, 32, 3)      \
  X(8, 2, 1, 16, 4)      \
  X(8, 1, 2, 32, 3)      \
  X(8, 1, 4, 16, 4)      \
  X(8, 1, 4, 24, 3)

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
cudaError_t launch_tmw9(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s);

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
    case Kind::TmW9:
      return launch_tmw9(cfg, dtype, a, s);

    case Kind::U8Pk:
      if (dtype != DD_U8_I32 || weighted) return cudaErrorInvalidConfiguration;
      return launch_u8pk(cfg, a, s);
  }
  return cudaErrorInvalidConfiguration;
}

// ------------------------------------------------------ persistent launches

int u8pk_smem_for(const TileConfig& cfg, int pitch);
int staged_smem_for(dd_dtype dtype, int stages, int cc, int bd, int pitch);

// The persistent kernel of a configuration (PERSISTENT) or its plain
// unweighted kernel, with its block size; null if there is none.
template <bool PERSISTENT>
static const void* kernel_of(const TileConfig& cfg, dd_dtype dtype, int* threads) {
  switch (cfg.kind) {
    case Kind::Staged:
      *threads = 256;
#define X(BD_, BT_, CC_, ST_)                                                                                   \
  if (cfg.bd == BD_ && cfg.bt == BT_ && cfg.cc == CC_ && cfg.stages == ST_) {                              \
    if (dtype == DD_U8_I32)                                                                                \
      return PERSISTENT ? (const void*)fwd_staged_persistent<uint8_t, false, BD_, BT_, CC_, ST_>           \
                        : (const void*)fwd_staged_kernel<uint8_t, false, BD_, BT_, CC_, ST_>;              \
    return PERSISTENT ? (const void*)fwd_staged_persistent<float, false, BD_, BT_, CC_, ST_>               \
                      : (const void*)fwd_staged_kernel<float, false, BD_, BT_, CC_, ST_>;                  \
  }
      DD_STAGED_CASES(X)
#undef X
      return nullptr;
    case Kind::U8Pk: {
      const int nw = cfg.threads / 32, wt = cfg.bt / (32 * 28), wd = nw / wt, dpw = cfg.bd / wd;
      *threads = cfg.threads;
#define X(WD_, WT_, DPW_, CC_, ST_)                                                                   \
  if (wd == WD_ && wt == WT_ && dpw == DPW_ && cfg.cc == CC_ && cfg.stages == ST_)                \
    return PERSISTENT ? (const void*)fwd_u8pk_persistent<WD_, WT_, DPW_, CC_, ST_>                 \
                      : (const void*)fwd_u8pk_kernel<WD_, WT_, DPW_, CC_, ST_>;
      DD_U8PK_CASES(X)
#undef X
      return nullptr;
    }
    case Kind::TmW9:
      *threads = cfg.threads;
      return PERSISTENT ? tmw9_persistent_kernel() : tmw9_plain_kernel();
    default:
      return nullptr;
  }
}

bool has_persistent(const TileConfig& cfg, dd_dtype dtype) {
  int threads = 0;
  return (cfg.kind == Kind::Staged || cfg.kind == Kind::U8Pk || cfg.kind == Kind::TmW9) &&
         kernel_of<true>(cfg, dtype, &threads) != nullptr;
}

int persistent_smem(const TileConfig& cfg, dd_dtype dtype, int pitch) {
  switch (cfg.kind) {
    case Kind::Staged: return staged_smem_for(dtype, cfg.stages, cfg.cc, cfg.bd, pitch);
    case Kind::U8Pk: return u8pk_smem_for(cfg, pitch);
    case Kind::TmW9: return cfg.smem;
    default: return 0;
  }
}

// Resident blocks per SM of a kernel at `smem` bytes of dynamic shared memory (0: cannot launch).
static int blocks_per_sm(const void* kern, int threads, int smem) {
  int per_sm = 0;
  if (!kern || cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess)
    return 0;
  return per_sm;
}

int persistent_blocks_per_sm(const TileConfig& cfg, dd_dtype dtype, int smem) {
  int threads = 0;
  const void* kern = kernel_of<true>(cfg, dtype, &threads);
  return blocks_per_sm(kern, threads, smem);
}

int plain_blocks_per_sm(const TileConfig& cfg, dd_dtype dtype, int smem) {
  int threads = 0;
  const void* kern = kernel_of<false>(cfg, dtype, &threads);
  return blocks_per_sm(kern, threads, smem);
}

cudaError_t launch_persistent(const TileConfig& cfg, dd_dtype dtype, const BatchWork& w, int smem, int grid,
                              cudaStream_t s) {
  if (w.n_items <= 0) return cudaSuccess;
  int threads = 0;
  const void* kern = kernel_of<true>(cfg, dtype, &threads);
  if (!kern || grid < 1) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  BatchWork arg = w;
  void* args[] = {&arg};
  return cudaLaunchKernel(kern, dim3(grid), dim3(threads), args, (size_t)smem, s);
}

std::vector<TileConfig> staged_menu(dd_dtype dtype) {
  std::vector<TileConfig> v;
  (void)dtype;
  // the generic kernel's block size is a launch parameter: four shapes
  v.push_back({Kind::Naive, 1, 256, 0, 0, 256, 0, 0, 0, "naive_t256"});
  v.push_back({Kind::Naive, 1, 128, 0, 0, 128, 0, 0, 0, "naive_t128"});
  v.push_back({Kind::Naive, 1, 64, 0, 0, 64, 0, 0, 0, "naive_t64"});
  v.push_back({Kind::Naive, 1, 32, 0, 0, 32, 0, 0, 0, "naive_t32"});
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
