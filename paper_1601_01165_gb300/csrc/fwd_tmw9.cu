// TMW9 forward kernel (float32): 9 DM trials x 4096 samples per block; each
// channel's input window sits in Tensor Memory once and serves all 9 trials.
//
// Section 2 notes that nearby DM trials read nearly the same input samples,
// and Section 2.2 shares a staged input span among the trials of a work
// group.  Here the span lives in Tensor Memory (TMEM), which a warp reads at a
// run-time column address (registers cannot be indexed at run time) faster
// than shared memory.  What bounds such a kernel is the copy of each window
// into TMEM: a 3-D TMA load writes the tile into shared memory, and the
// window goes shared -> registers -> TMEM.  Both copies use the SM's shared
// memory bandwidth, so the kernel shares every window among as many trials as
// the registers allow (9, against 6 in TMW6) and copies windows at 4-float
// granularity:
//
//  * TMEM lane r (quadrant q = r / 32 is also the reading warps' SM
//    sub-partition) holds the window of input that lane r's 32 output samples
//    need for the 9 trials of the block: samples [t0 + 32 r + d0, ... + 32 +
//    max offset), d0 = delay(c, i0), taken from the 4-float boundary at or
//    below its start.  Two sets of three 80-column slots hold the windows of
//    the current step of three channels and of the next one.
//  * Eight tensor maps view the input from float 4k (k = 0..7) in rows of 32
//    floats.  The map k = (t0 + d0) / 4 mod 8 puts the window's first 4-float
//    chunk at chunk 0 of tile row r, so a window is always chunks 0..n-1 of
//    rows r, r + 1, r + 2: compile-time shared addresses (128-byte swizzle,
//    conflict-free 16-byte loads), n = ceil(((d0 mod 4) + 32 + max offset) / 4).
//  * 12 warps, 3 per quadrant; warp p of a quadrant owns trials 3p..3p+2.
//    Per channel it reads its trials' 32 columns in six phases of 16
//    (tcgen05.ld.32x32b.x16, one trial per phase, trials in turn): it waits
//    for a phase's load, issues the next phase's, and adds the waited-for
//    values (packed pairs, add.rn.f32x2: two IEEE adds per instruction), so
//    every load is in flight during a phase of adds.  Trial columns come
//    straight from the block's descriptor row in global memory (L1-resident),
//    read a channel ahead and broadcast from lane 0, so the compiler keeps
//    the TMEM addresses in uniform registers: no cross-warp bookkeeping.
//  * Warp p writes the window of channel p of the next step while it works on
//    the step's last channel, from its private TMA stage (four 16-byte
//    chunks per 16-column TMEM store); it then reloads the stage with its
//    channel three later, so each tile load has one step to land.  (Deeper
//    staging, loads two or three steps ahead, ran slower: 2.66 and 2.69 ms
//    against 2.52 on the Apertif beam, whatever the shared-memory size; with
//    the copy moved from the step's middle channel to its last, 2.50.)
//  * The quadrant's three warps meet at a named barrier between steps, after
//    the last loads of the step have been waited for and before the next
//    step's first loads are issued: the next windows are then in TMEM and
//    this step's slots are free, and no load is stalled by the barrier.
//
// Stage-full mbarriers count the TMA bytes; every wait on them is bounded and
// a timeout sets the status word (the warps still run every step, so every
// named barrier completes).  Sums run over channels in ascending order as in
// every kernel here, so results are bit-identical to theirs.  The 9 x 4096
// sums leave through a swizzled shared-memory tile with 16-byte stores.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "dd_internal.h"
#include "ptx.cuh"

namespace dd {

namespace {

constexpr int kT = 9;                     // DM trials per block
constexpr int kTPW = 3;                   // trials per warp
constexpr int kQRows = 34;                // tile rows per quadrant: 32 lanes + 2 (a window spans <= 17 chunks)
constexpr int kTileBytes = kQRows * 128;  // 4352
constexpr int kStage = 5 * 1024;          // whole 1024-byte swizzle atoms
constexpr int kWS = 1;                    // stages per warp (its next own channel in flight)
constexpr int kSlot = 80;                 // columns per window slot (20 chunks)
constexpr int kLead = 3;                  // warps per quadrant = channels per step
constexpr int kAhead = kLead * kWS;       // a warp's tile loads run this many channels ahead
constexpr int kBT = 128 * 32;             // samples per block
constexpr int kThreads = 384;
constexpr int kHdr = 1024;
constexpr int kNStages = 12 * kWS;
constexpr int kOutTile = kT * kBT * 4;  // the epilogue's tile reuses the stage area
constexpr int kSmem = kHdr + (kNStages * kStage > kOutTile ? kNStages * kStage : kOutTile) +
                      1024;  // + slack to align the stages to 1024 bytes
constexpr uint32_t kCols = 512;
constexpr int kMaps = 8;
static_assert(2 * kLead * kSlot <= (int)kCols, "two sets of three windows fit TMEM");
static_assert(3 + kW9MaxOff + 32 <= kSlot, "a trial's 32 columns stay inside its window slot");
static_assert(4 * 20 <= kSlot, "five 4-chunk batches fit a slot");
static_assert((3 + 32 + kW9MaxOff + 3) / 4 <= 2 * 8 + 1, "a window spans rows r..r+2 of the tile");
static_assert(kTileBytes <= kStage, "stage holds the tile");
static_assert(kHdr + kOutTile + 1024 <= kSmem, "output tile fits the stage area");

struct Hdr {
  uint64_t sfull[12][kWS];  // per warp: its stages
  uint32_t tbase;
  int failed;
};
static_assert(sizeof(Hdr) <= kHdr, "header fits");

// Rows of a tile written by a 128B-swizzled TMA load (tile base 1024-byte
// aligned): 16-byte chunk x (0..7) of row y sits at y * 128 + ((x ^ y) & 7) * 16,
// which is rbase(y) ^ (x << 4) with rbase(y) = y * 128 + ((y & 7) << 4).
__device__ __forceinline__ uint32_t rbase(int y) { return (uint32_t)y * 128u + ((uint32_t)(y & 7) << 4); }

// Chunks X0..X0+3 of one tile row to 16 TMEM columns in one store.
template <int X0>
__device__ __forceinline__ void copy4(const unsigned char* tile, uint32_t rb, uint32_t taddr) {
  const float4 v0 = *reinterpret_cast<const float4*>(tile + (rb ^ (uint32_t)((X0 + 0) << 4)));
  const float4 v1 = *reinterpret_cast<const float4*>(tile + (rb ^ (uint32_t)((X0 + 1) << 4)));
  const float4 v2 = *reinterpret_cast<const float4*>(tile + (rb ^ (uint32_t)((X0 + 2) << 4)));
  const float4 v3 = *reinterpret_cast<const float4*>(tile + (rb ^ (uint32_t)((X0 + 3) << 4)));
  tmem_st16(taddr, v0, v1, v2, v3);
}

// Warp p's three trial columns (bytes 0..2 of word 1 + p of a descriptor),
// broadcast from lane 0 (the same for every lane).
__device__ __forceinline__ uint32_t warp_cols(const int4* d, int p) {
  return __shfl_sync(0xffffffffu, __ldg(reinterpret_cast<const uint32_t*>(d) + 1 + p), 0);
}

}  // namespace

// Eight views of the float input [C][in_stride], view k starting at float 4k:
// [C][rows_k][32], rows 128 bytes apart.
struct Tmw9Maps {
  CUtensorMap m[kMaps];
};

// Weight-gradient form of the tile (see fwd_tmw9_wgrad_kernel): grad_out
// [n_dm][g_stride] and the per-warp partial sums.
struct WgradArgs {
  const float* g;
  int64_t g_stride;
  float* partial;  // [C][n_part]: channel c's share from warp w of tile b at c * n_part + 12 b + w
  int64_t n_part;
};

// Load phases of one channel: six, each loading 16 columns of one trial
// (tcgen05.ld.32x32b.x16), trials in turn: phase f reads trial f % 3,
// columns 16 (f / 3) .. + 16.
constexpr int kPH = 16;
constexpr int kNPH = 6;
__device__ constexpr int ph_trial(int f) { return f % 3; }
__device__ constexpr int ph_col(int f) { return 16 * (f / 3); }

// Block set-up shared by the plain and the persistent kernel: the stage
// barriers, the status flag and the Tensor Memory allocation.
__device__ __forceinline__ void tmw9_setup(Hdr& H, int warp) {
  if (threadIdx.x == 0) {
    for (int w = 0; w < 12; ++w)
      for (int j = 0; j < kWS; ++j) mbar_init(&H.sfull[w][j], 1);
    H.failed = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&H.tbase, kCols);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
}

__device__ __forceinline__ void tmw9_teardown(Hdr& H, int warp) {
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(H.tbase, kCols);
}

// Own channels of warp p (channels c = p mod 3) among C.
__device__ __forceinline__ int own_channels(int C, int p) { return C > p ? (C - 1 - p) / kLead + 1 : 0; }

// One tile: trials [9 g, 9 g + 9) x samples [4096 ty, + 4096).  `mb` counts
// this warp's own channels of the block's earlier tiles (a persistent block
// runs tile after tile): the warp's m-th own channel of this tile is its
// (mb + m)-th, which fixes its stage and that stage's barrier phase.  False
// after a timeout (reported in the status word; no output written).  A
// block's last tile (LAST) frees the Tensor Memory as soon as the sums are in
// registers and skips the barrier that guards the stage area for a next tile.
template <bool WEIGHTED, bool LAST, bool GRADW = false>
__device__ __forceinline__ bool tmw9_tile(const Tmw9Maps& maps, const FwdArgs& a, int g, int ty, int mb, Hdr& H,
                                          unsigned char* stages, int warp, const WgradArgs* wg = nullptr,
                                          int tile = 0) {
  static_assert(!(GRADW && WEIGHTED), "the weight gradient does not use the weights");
  const int tid = threadIdx.x, lane = tid & 31;
  const int q = warp & 3, p = warp >> 2;
  const int r = 32 * q + lane;  // TMEM lane of this thread
  const int64_t t0 = (int64_t)ty * kBT;
  const int i0 = g * kT;
  const int C = a.C;
  const int4* gdesc = a.nine_desc + (int64_t)g * C;  // this block's descriptors, one per channel
  const uint32_t tq = __shfl_sync(0xffffffffu, H.tbase, 0) + ((uint32_t)(32 * q) << 16);  // quadrant's lanes, column 0

  // ------------------------------------------------ this warp's tile loads
  // Warp (q, p) writes the windows of channels c = p (mod 3) for quadrant q.
  // Its m-th channel (c = p + 3m) sits in stage m % kWS; lane 0 loads the
  // quadrant's 34 rows there and reloads the stage with channel c + 3 kWS
  // once the window is out.
  unsigned char* my_stages = stages + (size_t)warp * kWS * kStage;
  int issued = 0;  // own channels whose load was issued (lane 0)
  auto base_of = [&](int c) { return c < C ? __ldg(&gdesc[c].x) : 0; };
  auto issue = [&](int c, int base) {
    const int m = mb + (c - p) / kLead, j = m % kWS;
    unsigned char* st = my_stages + (size_t)j * kStage;
    const int64_t s0 = t0 + base;           // lane 0's first sample; its 4-float chunk starts the window
    const int k4 = (int)((s0 >> 2) & 7);    // the view whose rows start at that chunk
    mbar_arrive_expect_tx(&H.sfull[warp][j], kTileBytes);
    tma_load_3d(st, &maps.m[k4], 0, (int)(s0 >> 5) + 32 * q, c, &H.sfull[warp][j]);
  };
  int nbase = 0;  // base delay of this warp's next channel to load (lane 0)
  if (lane == 0) {
    int b0[kWS];
#pragma unroll
    for (int j = 0; j < kWS; ++j) b0[j] = base_of(p + kLead * j);
#pragma unroll
    for (int j = 0; j < kWS; ++j)
      if (p + kLead * j < C) {
        issue(p + kLead * j, b0[j]);
        ++issued;
      }
    nbase = base_of(p + kAhead);
  }

  // ------------------------------------------ window writer (one channel)
  // Copies the n-chunk window of channel c (c = p mod 3) from this warp's
  // stage into slot p of set `set` and reloads the stage; false on a timeout
  // (the window is then left unwritten and the block reports the error).
  auto write_window = [&](int c, int set) -> bool {
    const int m = mb + (c - p) / kLead, j = m % kWS;
    const int nch = __shfl_sync(0xffffffffu, (int)((uint32_t)__ldg(&gdesc[c].y) >> 24), 0);
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&H.sfull[warp][j], (uint32_t)((m / kWS) & 1), kWaitLimitCycles)))
      return false;
    const unsigned char* st = my_stages + (size_t)j * kStage;
    const uint32_t col = tq + (uint32_t)(kSlot * (kLead * set + p));
    if (DD_INDEX_OK(a.status, nch >= 8 && nch <= 17 && lane + 2 < kQRows)) {
      // chunk k of the window is chunk k & 7 of tile row lane + (k >> 3)
      const uint32_t rb0 = rbase(lane), rb1 = rbase(lane + 1);
      copy4<0>(st, rb0, col);
      copy4<4>(st, rb0, col + 16);
      if (nch > 8) copy4<0>(st, rb1, col + 32);
      if (nch > 12) copy4<4>(st, rb1, col + 48);
      if (nch > 16) copy4<0>(st, rbase(lane + 2), col + 64);
    }
    __syncwarp();
    if (lane == 0) {
      // the stage is read (the TMEM stores consumed the shared loads): reload
      // it with this warp's channel kAhead later
      if (c + kAhead < C) {
        issue(c + kAhead, nbase);
        ++issued;
        nbase = base_of(c + kAhead + kLead);
      }
    }
    return true;
  };
  // The quadrant's three warps meet at a named barrier between steps.  Every
  // warp runs the same channels whatever happens (a timeout only skips
  // work), so each barrier is always completed.
  const uint32_t bar_id = 1 + (uint32_t)q;
  auto quad_sync = [&]() {
    tmem_wait_st();
    tmem_fence_before_sync();
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(32 * kLead) : "memory");
    tmem_fence_after_sync();
  };
  // TMEM address of this warp's trial jj in a slot (columns checked in
  // checked builds: the 32 columns stay inside the slot)
  auto trial_addr = [&](uint32_t slot_col, uint32_t cols, int jj) -> uint32_t {
    uint32_t o = (cols >> (8 * jj)) & 0xffu;
    if (!DD_INDEX_OK(a.status, o + 32 <= (uint32_t)kSlot)) o = 0;
    return slot_col + o;
  };

  bool ok = true;
  if (p < C) ok = write_window(p, 0);  // step 0's windows go to set 0
  quad_sync();

  // ------------------------------------------------------------ main loop
  // forward: acc holds the sums; weight gradient: acc holds this thread's
  // grad_out values (zero outside the output), and s the channel's products
  float acc[kTPW][32];
  float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;  // two independent pairs: shorter add chains
  float vstep[kLead];  // the step's channels' per-lane products (weight gradient)
  int nl = 32;            // this lane's samples inside the output (weight gradient)
  bool mask_lane = false;  // warp-uniform: this tile holds a lane that ends inside the output
  if constexpr (GRADW) {
    const int64_t tl = t0 + 32 * r;
    nl = (int)max((int64_t)0, min((int64_t)32, a.n_out - tl));
    mask_lane = t0 + kBT > a.n_out && a.n_out % 32 != 0;
    const bool vec = (reinterpret_cast<uintptr_t>(wg->g) % 16 == 0) && (wg->g_stride % 4 == 0) && nl == 32;
#pragma unroll
    for (int jj = 0; jj < kTPW; ++jj) {
      const int i = i0 + kTPW * p + jj;
      const float* gr = wg->g + (int64_t)min(i, a.n_dm - 1) * wg->g_stride + tl;
      if (vec && i < a.n_dm) {
#pragma unroll
        for (int k4 = 0; k4 < 8; ++k4) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(gr) + k4);
          acc[jj][4 * k4] = v.x, acc[jj][4 * k4 + 1] = v.y, acc[jj][4 * k4 + 2] = v.z, acc[jj][4 * k4 + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[jj][k] = (i < a.n_dm && k < nl) ? __ldg(gr + k) : 0.0f;
      }
    }
  } else {
#pragma unroll
    for (int jj = 0; jj < kTPW; ++jj)
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[jj][k] = 0.0f;
  }
  float X[kPH], Y[kPH];
  uint32_t ta[kTPW];
  float wc = 1.0f;
  if constexpr (WEIGHTED) wc = __ldg(a.w);
  {
    const uint32_t cols = warp_cols(gdesc, p);
#pragma unroll
    for (int jj = 0; jj < kTPW; ++jj) ta[jj] = trial_addr(tq, cols, jj);
    tmem_ld16(ta[ph_trial(0)] + ph_col(0), X);
  }
  const int n_steps = (C + kLead - 1) / kLead;
#pragma unroll 1
  for (int n = 0; n < n_steps; ++n) {
    const int set = n & 1;
#pragma unroll
    for (int k = 0; k < kLead; ++k) {
      const int c = kLead * n + k;
      if (c >= C) break;  // the same for every warp
      // the next channel's trial columns and weight, a channel ahead
      const bool more = c + 1 < C;
      const uint32_t cols_n = more ? warp_cols(gdesc + c + 1, p) : 0u;
      float wn = 1.0f;
      if constexpr (WEIGHTED) wn = more ? __ldg(a.w + c + 1) : wc;
#pragma unroll
      for (int f = 0; f < kNPH; ++f) {
        float* cur = (f & 1) ? Y : X;
        float* nxt = (f & 1) ? X : Y;
        tmem_wait_ld16(cur);
        if (f + 1 < kNPH) {
          tmem_ld16(ta[ph_trial(f + 1)] + ph_col(f + 1), nxt);
        } else if (more) {
          // the next channel; at a step boundary the next windows must be in
          // place and this step's slots free first
          if (k == kLead - 1) quad_sync();
          const int nset = k == kLead - 1 ? set ^ 1 : set;
          const int nk = k == kLead - 1 ? 0 : k + 1;
          const uint32_t slot_col = tq + (uint32_t)(kSlot * (kLead * nset + nk));
#pragma unroll
          for (int jj = 0; jj < kTPW; ++jj) ta[jj] = trial_addr(slot_col, cols_n, jj);
          tmem_ld16(ta[ph_trial(0)] + ph_col(0), nxt);
        }
        if constexpr (GRADW) {
          const int jj = ph_trial(f), c0 = ph_col(f);
          if (mask_lane) {
            // in the lane that holds the output's last samples, the samples
            // past the output read input past n_in (padding the caller owns,
            // maybe not finite): they must not reach the sum
#pragma unroll
            for (int u = 0; u < kPH; ++u) cur[u] = c0 + u < nl ? cur[u] : 0.0f;
          }
#pragma unroll
          for (int u = 0; u < kPH; u += 4) {
            fma2v_rn(s0, s1, cur[u], cur[u + 1], acc[jj][c0 + u], acc[jj][c0 + u + 1]);
            fma2v_rn(s2, s3, cur[u + 2], cur[u + 3], acc[jj][c0 + u + 2], acc[jj][c0 + u + 3]);
          }
          if (f == kNPH - 1) {
            // the warp's shares of the step's channels, reduced together at
            // the step's end (interleaved, in a fixed order) and stored by lane 0
            vstep[k] = nl > 0 ? (s0 + s1) + (s2 + s3) : 0.0f;  // lanes past the output add nothing
            s0 = s1 = s2 = s3 = 0.0f;
            if (k == kLead - 1 || !more) {
#pragma unroll
              for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int kk = 0; kk <= k; ++kk) vstep[kk] += __shfl_xor_sync(0xffffffffu, vstep[kk], o);
              if (lane == 0) {
#pragma unroll
                for (int kk = 0; kk <= k; ++kk)
                  wg->partial[(int64_t)(c - k + kk) * wg->n_part + (int64_t)tile * 12 + warp] = vstep[kk];
              }
            }
          }
        } else {
          const int jj = ph_trial(f), c0 = ph_col(f);
#pragma unroll
          for (int u = 0; u < kPH; u += 2) {
            float& a0 = acc[jj][c0 + u];
            float& a1 = acc[jj][c0 + u + 1];
            if constexpr (WEIGHTED)
              fma2_rn(a0, a1, wc, cur[u], cur[u + 1]);
            else
              add2_rn(a0, a1, cur[u], cur[u + 1]);
          }
        }
        // this warp's window of the next step, while a phase's load is in
        // flight (all warps at the same point of the step)
        if (f == 1 && k == kLead - 1 && ok) {
          const int cw = kLead * (n + 1) + p;
          if (cw < C) ok = write_window(cw, set ^ 1);
        }
      }
      wc = wn;
    }
  }
  if (!ok && lane == 0) {
    report_error(a.status, kDevWaitTimeout);
    atomicExch(&H.failed, 1);
  }
  tmem_wait_st();
  tmem_wait_ld();
  // no TMA may still be landing when the stage area is reused or the block
  // leaves (after a timeout some loads may not have been consumed)
  if (lane == 0) {
    for (int m = mb + max(0, issued - kWS); m < mb + issued; ++m)
      (void)mbar_wait_bounded(&H.sfull[warp][m % kWS], (uint32_t)((m / kWS) & 1), kWaitLimitCycles);
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (LAST && warp == 0) tmem_dealloc(H.tbase, kCols);
  if (H.failed) return false;
  if constexpr (GRADW) return true;  // the partials are out

  // ------------------------------------------------------------ epilogue
  // trial-major tile of 16-byte chunks; chunk k4 of row r sits at k4 ^ (r & 7)
  float4* ot = reinterpret_cast<float4*>(stages);
#pragma unroll
  for (int jj = 0; jj < kTPW; ++jj) {
    float4* row = ot + (size_t)(kTPW * p + jj) * (kBT / 4) + r * 8;
#pragma unroll
    for (int k4 = 0; k4 < 8; ++k4)
      row[k4 ^ (r & 7)] = make_float4(acc[jj][4 * k4], acc[jj][4 * k4 + 1], acc[jj][4 * k4 + 2], acc[jj][4 * k4 + 3]);
  }
  __syncthreads();
  float* __restrict__ out = static_cast<float*>(a.out);
  const bool vec = (reinterpret_cast<uintptr_t>(out) % 16 == 0) && (a.out_stride % 4 == 0);
  for (int u = tid; u < kT * (kBT / 4); u += kThreads) {
    const int j = u / (kBT / 4), m = u % (kBT / 4);
    const int i = i0 + j;
    if (i >= a.n_dm) break;  // u grows with j
    const int rr = m >> 3, k4 = m & 7;
    const float4 x = ot[(size_t)j * (kBT / 4) + rr * 8 + (k4 ^ (rr & 7))];
    const int64_t t = t0 + 4 * m;
    float* o = out + (int64_t)i * a.out_stride + t;
    if (vec && t + 3 < a.n_out) {
      *reinterpret_cast<float4*>(o) = x;
    } else {
      if (t < a.n_out) o[0] = x.x;
      if (t + 1 < a.n_out) o[1] = x.y;
      if (t + 2 < a.n_out) o[2] = x.z;
      if (t + 3 < a.n_out) o[3] = x.w;
    }
  }
  // the next tile of a persistent block loads into this area again
  if (!LAST) __syncthreads();
  return true;
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kThreads, 1) fwd_tmw9_kernel(const __grid_constant__ Tmw9Maps maps, FwdArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Hdr& H = *reinterpret_cast<Hdr*>(smem_raw);
  const uint32_t sbase = smem_u32(smem_raw);
  unsigned char* stages = smem_raw + (((sbase + kHdr + 1023u) & ~1023u) - sbase);
  // warp-uniform values go through a lane-0 broadcast, which lets the
  // compiler keep them (and the TMEM addresses built from them) in uniform
  // registers instead of moving each address over before each TMEM access
  const int warp = __shfl_sync(0xffffffffu, (int)threadIdx.x >> 5, 0);
  tmw9_setup(H, warp);
  (void)tmw9_tile<WEIGHTED, true>(maps, a, blockIdx.x, blockIdx.y, 0, H, stages, warp);
}

// Weight gradient of the forward (grad_w[c] = sum_i sum_t grad_out[i][t]
// in[c][t + d(c, i)]) on the forward's tiles: each thread keeps its 96
// grad_out values where the forward keeps its sums, multiplies them with the
// same Tensor-Memory windows and adds the products of each channel; every
// warp stores its share of each channel's sum (a fixed-order shuffle
// reduction), and wgrad_reduce_kernel adds the shares in a fixed order.
__global__ void __launch_bounds__(kThreads, 1)
    fwd_tmw9_wgrad_kernel(const __grid_constant__ Tmw9Maps maps, FwdArgs a, WgradArgs wg) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Hdr& H = *reinterpret_cast<Hdr*>(smem_raw);
  const uint32_t sbase = smem_u32(smem_raw);
  unsigned char* stages = smem_raw + (((sbase + kHdr + 1023u) & ~1023u) - sbase);
  const int warp = __shfl_sync(0xffffffffu, (int)threadIdx.x >> 5, 0);
  tmw9_setup(H, warp);
  const int tile = (int)(blockIdx.y * gridDim.x + blockIdx.x);
  (void)tmw9_tile<false, true, true>(maps, a, blockIdx.x, blockIdx.y, 0, H, stages, warp, &wg, tile);
}

// grad_w[c] = the sum of channel c's n_part shares: one block per channel,
// each thread a strided subset in double, then a fixed reduction tree.
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(const float* __restrict__ partial, int64_t n_part,
                                                          float* __restrict__ grad_w) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  const float* row = partial + (int64_t)c * n_part;
  double sum = 0.0;
  for (int64_t k = threadIdx.x; k < n_part; k += 256) sum += (double)row[k];
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad_w[c] = (float)red[0];
}

// Persistent form for batches: the block takes tiles of many beams from the
// work list (see BatchWork; each beam's eight views sit in w.maps) until it is
// exhausted; its Tensor Memory, stages and barriers carry over from tile to
// tile.
__global__ void __launch_bounds__(kThreads, 1) fwd_tmw9_persistent(const __grid_constant__ BatchWork w) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Hdr& H = *reinterpret_cast<Hdr*>(smem_raw);
  const uint32_t sbase = smem_u32(smem_raw);
  unsigned char* stages = smem_raw + (((sbase + kHdr + 1023u) & ~1023u) - sbase);
  const int warp = __shfl_sync(0xffffffffu, (int)threadIdx.x >> 5, 0);
  __shared__ int item_s;
  tmw9_setup(H, warp);
  int mb = 0;
  while (true) {
    WorkItem it;
    if (!next_item(w, item_s, it)) break;
    const BatchBeam& bm = w.beams[it.beam];  // kernel parameters
    const Tmw9Maps& maps = static_cast<const Tmw9Maps*>(w.maps)[it.beam];
    // the beam's views live in global memory: fetch them before the first loads
    if (threadIdx.x < kMaps) prefetch_tensormap(&maps.m[threadIdx.x]);
    const bool ok = tmw9_tile<false, false>(maps, bm.a, it.x, it.y, mb, H, stages, warp);
    mb += own_channels(bm.a.C, warp >> 2);
    if (__syncthreads_or(!ok)) break;
  }
  tmw9_teardown(H, warp);
}

// ------------------------------------------------------------------- launch

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
static EncodeTiledFn encode_fn9() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Rows of view k: whole 32-float rows from float 4k of `in` to the end of
// the channel's row (`avail` elements from `in`).
static int64_t view_rows(int64_t avail, int k) { return (avail - 4 * k) / 32; }

// `avail` = elements from `in` to the end of each row (the stride, less the
// first sample of a time-chunked launch).
static bool tmw9_accepts_avail(const void* in, int64_t in_stride, int64_t avail, int64_t n_in) {
  if ((reinterpret_cast<uintptr_t>(in) % 16) != 0 || in_stride % 4 != 0 || encode_fn9() == nullptr) return false;
  // every sample a valid output can need (index < n_in) lies in a whole row of
  // every view: the views end at the last whole row inside the channel's row
  for (int k = 0; k < kMaps; ++k) {
    const int64_t rows = view_rows(avail, k);
    if (rows < 1 || n_in - 1 - 4 * k >= 32 * rows) return false;
  }
  return true;
}

bool tmw9_accepts(const void* in, int64_t in_stride, int64_t n_in) {
  return tmw9_accepts_avail(in, in_stride, in_stride, n_in);
}

int64_t tmw9_min_in_stride(int64_t n_in) {
  // a multiple of 32 floats with at least 28 to spare keeps the last needed
  // sample inside view 1..7's last whole row
  return (n_in + 28 + 31) / 32 * 32;
}

static bool encode_views(Tmw9Maps* maps, const FwdArgs& a) {
  EncodeTiledFn fn = encode_fn9();
  if (!fn) return false;
  for (int k = 0; k < kMaps; ++k) {
    const cuuint64_t dims[3] = {32, (cuuint64_t)view_rows(a.in_avail, k), (cuuint64_t)a.C};
    const cuuint64_t strides[2] = {128, (cuuint64_t)a.in_stride * 4};
    const cuuint32_t box[3] = {32, (cuuint32_t)kQRows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    void* base = const_cast<float*>(static_cast<const float*>(a.in) + 4 * k);
    if (fn(&maps->m[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

cudaError_t launch_tmw9(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s) {
  (void)cfg;
  if (dtype != DD_F32_F32) return cudaErrorInvalidConfiguration;
  if (a.nine_desc == nullptr || !tmw9_accepts_avail(a.in, a.in_stride, a.in_avail, a.n_in))
    return cudaErrorInvalidConfiguration;
  Tmw9Maps maps;
  if (!encode_views(&maps, a)) return cudaErrorInvalidValue;
  auto kern = a.w ? fwd_tmw9_kernel<true> : fwd_tmw9_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((a.n_dm + kT - 1) / kT), (unsigned)((a.n_out + kBT - 1) / kBT));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  kern<<<grid, kThreads, kSmem, s>>>(maps, a);
  return cudaGetLastError();
}

int64_t tmw9_wgrad_partials(const FwdArgs& a) {
  if (a.nine_desc == nullptr || !tmw9_accepts_avail(a.in, a.in_stride, a.in_avail, a.n_in)) return 0;
  const int64_t tiles = (int64_t)((a.n_dm + kT - 1) / kT) * ((a.n_out + kBT - 1) / kBT);
  return tiles * 12 * a.C;
}

cudaError_t launch_tmw9_wgrad(const FwdArgs& a, const float* g, int64_t g_stride, float* partial, float* grad_w,
                              cudaStream_t s) {
  const int64_t n = tmw9_wgrad_partials(a);
  if (n <= 0 || g == nullptr || partial == nullptr || grad_w == nullptr) return cudaErrorInvalidConfiguration;
  Tmw9Maps maps;
  if (!encode_views(&maps, a)) return cudaErrorInvalidValue;
  auto kern = fwd_tmw9_wgrad_kernel;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((a.n_dm + kT - 1) / kT), (unsigned)((a.n_out + kBT - 1) / kBT));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  const int64_t n_part = n / a.C;
  kern<<<grid, kThreads, kSmem, s>>>(maps, a, WgradArgs{g, g_stride, partial, n_part});
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wgrad_reduce_kernel<<<a.C, 256, 0, s>>>(partial, n_part, grad_w);
  return cudaGetLastError();
}

size_t tmw9_views_bytes() { return sizeof(Tmw9Maps); }

bool tmw9_encode_views(const FwdArgs& a, void* out) {
  if (a.nine_desc == nullptr || !tmw9_accepts_avail(a.in, a.in_stride, a.in_avail, a.n_in)) return false;
  return encode_views(static_cast<Tmw9Maps*>(out), a);
}

const void* tmw9_persistent_kernel() { return (const void*)fwd_tmw9_persistent; }
const void* tmw9_plain_kernel() { return (const void*)fwd_tmw9_kernel<false>; }

std::vector<TileConfig> tmw9_menu(dd_dtype dtype) {
  std::vector<TileConfig> v;
  if (dtype != DD_F32_F32) return v;
  v.push_back({Kind::TmW9, kT, kBT, 1, kWS, kThreads, 32, kSmem, 0, "tmw9_f32_d9_t4096"});
  return v;
}

}  // namespace dd
