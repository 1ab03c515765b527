// TMW6 forward kernel (float32): 6 DM trials x 4096 samples per block, input
// windows shared through Tensor Memory, one batched TMEM read per channel.
//
// Section 2 notes that nearby DM trials read nearly the same input samples;
// Section 2.2 exploits it by sharing staged input within a work group.  Here
// the sharing happens in Tensor Memory, which a warp can read at a run-time
// column address (registers cannot be indexed at run time) and which returns
// values to registers several times faster than shared memory:
//
//  * TMEM lane r holds, per channel, the window of the input that lane r's 32
//    output samples need for all 6 trials: 32 + max offset columns, taken as
//    whole 16-float groups of the tile.  Two sets of three 80-column slots
//    hold the current step's windows and the next step's.
//  * 12 warps, 3 per TMEM lane quadrant (warp w serves lanes 32 (w % 4) ..,
//    which is also its SM sub-partition); warp p = w / 4 owns trials 2p and
//    2p + 1.  Each channel it reads its slot entry (its two trials' TMEM
//    addresses: the slot's column plus shift + o_j, o_j = delay(c, i0 + j) -
//    delay(c, i0), and the channel weight), issues two 32-column loads and
//    waits once; 32 packed adds (two IEEE adds per instruction) follow.
//  * Warp p of a quadrant writes the quadrant's window of channel p of the
//    next step of three channels, while its TMEM loads of the step's last
//    channel are in flight.  The input comes from its private stages: a 3-D
//    TMA load (128-byte swizzle) of the quadrant's 35 rows of 32 samples from
//    the row holding t0 + delay(c, i0), plus the channel's 16-byte descriptor
//    (base delay, column bytes, window width); 16-byte shared loads read the
//    swizzled rows without bank conflicts, each going straight to 4 TMEM
//    columns.  Three lanes then publish the reading warps' slot entries.
//    Once a window is out, the warp reloads the stage with its channel nine
//    later, so quadrants never wait on each other.
//  * The quadrant's three warps meet at a named barrier after each step: the
//    next step's windows are then in TMEM and this step's slots are free.
//
// Stage-full mbarriers count the TMA bytes; every wait on them is bounded and
// a timeout sets the status word (the warps still run every step, so every
// named barrier completes).  Sums run in channel order as in every kernel
// here, so results are bit-identical to theirs.  The 6 x 4096 sums leave
// through a swizzled shared-memory tile with coalesced 16-byte stores.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "dd_internal.h"
#include "ptx.cuh"

namespace dd {

namespace {

constexpr int kT = 6;                       // DM trials per block
constexpr int kQRows = 35;                  // tile rows of 32 samples per quadrant (32 lanes + 3)
constexpr int kTileBytes = kQRows * 128;    // 4480
constexpr int kStage = 5 * 1024;            // tile + descriptor, whole 1024-byte swizzle atoms
constexpr int kWS = 3;                      // stages per warp (its channels c, c + 3, c + 6 in flight)
constexpr int kSlot = 80;                   // columns per window: 5 groups of 16 (see the window writer)
constexpr int kLead = 3;                    // warps per quadrant = channels per step
constexpr int kAhead = kLead * kWS;         // a warp's tile loads run this many channels ahead
constexpr int kBT = 128 * 32;               // samples per block
constexpr int kThreads = 384;
constexpr int kHdr = 2048;
constexpr int kNStages = 12 * kWS;
constexpr int kSmem = kHdr + kNStages * kStage + 1024;  // + slack to align the stages to 1024 bytes
constexpr uint32_t kCols = 512;
static_assert(2 * 3 * kSlot <= (int)kCols, "two sets of three windows fit TMEM");
static_assert(12 + 3 + 32 + kW6MaxOff <= kSlot - 1, "a trial's last column stays inside its window");
static_assert(kTileBytes + 16 <= kStage, "stage holds tile and descriptor");
static_assert(kT * kBT * 4 <= kNStages * kStage, "output tile fits the stage area");

struct Hdr {
  uint64_t sfull[12][kWS];           // per warp: its stages
  uint4 slot[4][2 * kLead][kLead];   // per quadrant window slot and reading warp: its 2 trials' TMEM addresses, weight bits
  uint32_t tbase;
  int failed;
};
static_assert(sizeof(Hdr) <= kHdr, "header fits");

// Rows of a tile written by a 128B-swizzled TMA load (tile base 1024-byte
// aligned): 16-byte chunk x (0..7) of row y sits at y * 128 + ((x ^ y) & 7) * 16,
// which is rbase(y) ^ (x << 4) with rbase(y) = y * 128 + ((y & 7) << 4).
__device__ __forceinline__ uint32_t rbase(int y) { return (uint32_t)y * 128u + ((uint32_t)(y & 7) << 4); }

// One 16-byte chunk of each lane's row to 4 TMEM columns.
__device__ __forceinline__ void st4(uint32_t taddr, float4 x) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "f"(x.x), "f"(x.y),
               "f"(x.z), "f"(x.w));
}

// Four consecutive chunks of one row (compile-time chunk index X0..X0+3),
// each stored to TMEM as it arrives.
template <int X0>
__device__ __forceinline__ void copy_group(const unsigned char* tile, uint32_t rb, uint32_t taddr) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    st4(taddr + 4 * k, *reinterpret_cast<const float4*>(tile + (rb ^ (uint32_t)((X0 + k) << 4))));
}

}  // namespace

template <bool WEIGHTED>
__global__ void __launch_bounds__(kThreads, 1) fwd_tmw6_kernel(const __grid_constant__ CUtensorMap tmap, FwdArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Hdr& H = *reinterpret_cast<Hdr*>(smem_raw);
  // stages on the first 1024-byte boundary (of the shared address) past the
  // header; indexing the shared array keeps every access a shared one
  const uint32_t sbase = smem_u32(smem_raw);
  unsigned char* stages = smem_raw + (((sbase + kHdr + 1023u) & ~1023u) - sbase);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, p = warp >> 2;
  const int r = 32 * q + lane;  // TMEM lane of this thread
  // trial groups vary fastest: blocks resident together share one stretch of
  // the input, which then stays in L2
  const int64_t t0 = (int64_t)blockIdx.y * kBT;
  const int g = blockIdx.x;
  const int i0 = g * kT;
  const int C = a.C;
  const int4* gdesc = a.hex_desc + (int64_t)g * C;  // this block's descriptors, one per channel

  if (tid == 0) {
    for (int w = 0; w < 12; ++w)
      for (int j = 0; j < kWS; ++j) mbar_init(&H.sfull[w][j], 1);
    H.failed = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&H.tbase, kCols);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tq = H.tbase + ((uint32_t)(32 * q) << 16);  // this quadrant's lanes, column 0
  // slots start with in-range addresses (column 0 of the slot) and unit weight,
  // so a window left unwritten after a timeout is never read out of range
  if (lane == 0)
    for (int sl = p; sl < 2 * kLead; sl += kLead)
      for (int pr = 0; pr < kLead; ++pr) {
        const uint32_t c0 = tq + (uint32_t)(kSlot * sl);
        H.slot[q][sl][pr] = make_uint4(c0, c0, __float_as_uint(1.0f), 0u);
      }

  // ------------------------------------------------ this warp's tile loads
  // Warp (q, p) writes the windows of channels c = p (mod 3) for quadrant q.
  // Its m-th channel (c = p + 3m) sits in its stage m % kWS; lane 0 loads the
  // quadrant's 35 rows of the tile and the channel's descriptor there, and
  // reloads the stage with channel c + 9 once the window is out.
  unsigned char* my_stages = stages + (size_t)warp * kWS * kStage;
  int issued = 0;  // own channels whose load was issued (lane 0)
  auto base_of = [&](int c) { return c < C ? __ldg(&gdesc[c].x) : 0; };
  auto issue = [&](int c, int base) {
    const int m = (c - p) / kLead, j = m % kWS;
    unsigned char* st = my_stages + (size_t)j * kStage;
    mbar_arrive_expect_tx(&H.sfull[warp][j], kTileBytes + 16);
    bulk_g2s(st + kTileBytes, gdesc + c, 16, &H.sfull[warp][j]);
    tma_load_3d(st, &tmap, 0, (int)((t0 + base) >> 5) + 32 * q, c, &H.sfull[warp][j]);
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
  // Copies the window of channel c (c = p mod 3) from this warp's stage into
  // TMEM slot `sl` of the quadrant and reloads the stage; false on a timeout
  // (the window is then left unwritten and the block reports the error).
  auto write_window = [&](int c, int sl) -> bool {
    const int m = (c - p) / kLead, j = m % kWS;
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&H.sfull[warp][j], (uint32_t)((m / kWS) & 1), kWaitLimitCycles)))
      return false;
    unsigned char* st = my_stages + (size_t)j * kStage;
    const int4 dsc = *reinterpret_cast<const int4*>(st + kTileBytes);
    // The window is the 16-float groups of rows lane .. lane + 2 (96 floats)
    // that hold elements [4 c4, 4 c4 + need): groups G0 = c4 / 4 .. G0 + ng - 1,
    // stored from the slot's first column, so element 4 c4 + x lands on column
    // 4 (c4 % 4) + x.  G0 is 0 or 1: both cases use compile-time chunk indices.
    const int c4 = (int)((t0 + dsc.x) & 31) >> 2;
    const int need = dsc.w;  // floats from the aligned start: shift + 32 + max offset
    const int lead = 4 * (c4 & 3);
    const int ng = (lead + need + 15) >> 4;  // 3..5
    const uint32_t col = tq + (uint32_t)(kSlot * sl);
    // the window's groups stay inside the slot and the tile's rows
    if (!DD_INDEX_OK(a.status, need >= 32 && lead + need <= kSlot && lane + 2 < kQRows)) return true;
    const uint32_t rb0 = rbase(lane), rb1 = rbase(lane + 1), rb2 = rbase(lane + 2);
    if (c4 < 4) {  // groups 0..4: row lane (0, 1), row lane + 1 (2, 3), row lane + 2 (4)
      copy_group<0>(st, rb0, col);
      copy_group<4>(st, rb0, col + 16);
      copy_group<0>(st, rb1, col + 32);
      if (ng > 3) copy_group<4>(st, rb1, col + 48);
      if (ng > 4) copy_group<0>(st, rb2, col + 64);
    } else {  // groups 1..5
      copy_group<4>(st, rb0, col);
      copy_group<0>(st, rb1, col + 16);
      copy_group<4>(st, rb1, col + 32);
      if (ng > 3) copy_group<0>(st, rb2, col + 48);
      if (ng > 4) copy_group<4>(st, rb2, col + 64);
    }
    float wc = 1.0f;
    if constexpr (WEIGHTED) wc = __ldg(a.w + c);
    // lane pr < 3 publishes reading warp pr's entry: its trials' TMEM addresses
    // (the slot's column, the window's lead and the trial's column byte; the 32
    // columns stay inside the slot) and the channel's weight
    if (lane < kLead) {
      const uint32_t bytes = (uint32_t)(lane < 2 ? dsc.y : dsc.z) >> (16 * (lane & 1));
      uint32_t b0 = (uint32_t)lead + (bytes & 0xffu), b1 = (uint32_t)lead + ((bytes >> 8) & 0xffu);
      if (!DD_INDEX_OK(a.status, b0 + 32 <= (uint32_t)kSlot && b1 + 32 <= (uint32_t)kSlot)) b0 = b1 = 0;
      H.slot[q][sl][lane] = make_uint4(col + b0, col + b1, __float_as_uint(wc), 0u);
    }
    __syncwarp();
    if (lane == 0) {
      // the stage is read: reload it with this warp's channel kAhead later
      // (the window's shared loads have completed: the TMEM stores consumed them)
      if (c + kAhead < C) {
        issue(c + kAhead, nbase);
        ++issued;
        nbase = base_of(c + kAhead + kLead);
      }
    }
    return true;
  };
  // The quadrant's three warps meet at a named barrier once per step of three
  // channels.  Every warp runs the same number of steps whatever happens
  // (a timeout only skips work), so each barrier is always completed.
  const uint32_t bar_id = 1 + (uint32_t)q;
  auto quad_sync = [&]() {
    tmem_wait_st();
    tmem_fence_before_sync();
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(96) : "memory");
    tmem_fence_after_sync();
  };

  bool ok = true;
  if (p < C) ok = write_window(p, p);  // step 0's windows go to slots 0..2
  quad_sync();

  // ------------------------------------------------------------ main loop
  float acc[2][32];
#pragma unroll
  for (int jj = 0; jj < 2; ++jj)
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[jj][k] = 0.0f;
  const int n_steps = (C + kLead - 1) / kLead;
#pragma unroll 2
  for (int n = 0; n < n_steps; ++n) {
    const int set = (n & 1) * kLead;  // slots of this step's windows
#pragma unroll
    for (int k = 0; k < kLead; ++k) {
      const int c = kLead * n + k;
      if (c >= C) break;  // the same for every warp
      const uint4 ta = H.slot[q][set + k][p];  // trials 2p, 2p + 1 and the channel's weight
      float v0[32], v1[32];
      tmem_ld32(ta.x, v0);
      tmem_ld32(ta.y, v1);
      // while the step's last loads are in flight: this warp's window of the next step
      if (k == kLead - 1 && ok) {
        const int cn = kLead * (n + 1) + p;
        if (cn < C) ok = write_window(cn, (kLead - set) + p);
      }
      tmem_wait_ld();
      // packed pairs: half the add instructions of scalar code, same results
      if constexpr (WEIGHTED) {
        const float wc = __uint_as_float(ta.z);
#pragma unroll
        for (int u = 0; u < 32; u += 2) {
          fma2_rn(acc[0][u], acc[0][u + 1], wc, v0[u], v0[u + 1]);
          fma2_rn(acc[1][u], acc[1][u + 1], wc, v1[u], v1[u + 1]);
        }
      } else {
#pragma unroll
        for (int u = 0; u < 32; u += 2) {
          add2_rn(acc[0][u], acc[0][u + 1], v0[u], v0[u + 1]);
          add2_rn(acc[1][u], acc[1][u + 1], v1[u], v1[u + 1]);
        }
      }
    }
    quad_sync();  // next step's windows written; this step's slots free
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
    for (int m = max(0, issued - kWS); m < issued; ++m)
      (void)mbar_wait_bounded(&H.sfull[warp][m % kWS], (uint32_t)((m / kWS) & 1), kWaitLimitCycles);
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(H.tbase, kCols);
  if (H.failed) return;

  // ------------------------------------------------------------ epilogue
  // trial-major tile of 16-byte chunks; chunk k4 of row r sits at k4 ^ (r & 7)
  float4* ot = reinterpret_cast<float4*>(stages);
#pragma unroll
  for (int jj = 0; jj < 2; ++jj) {
    float4* row = ot + (size_t)(2 * p + jj) * (kBT / 4) + r * 8;
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
}

// ------------------------------------------------------------------- launch

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
static EncodeTiledFn encode_fn() {
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

bool tmw6_accepts(const void* in, int64_t in_stride) {
  return in_stride % 32 == 0 && (reinterpret_cast<uintptr_t>(in) % 16) == 0 && encode_fn() != nullptr;
}

// Tensor map over the float input viewed as [C][in_avail / 32 rows][32]: one
// load brings `rows` consecutive 128-byte rows of one channel, stored with
// the 128-byte swizzle; rows past the end of the channel's row (measured from
// `in`, which a time-chunked launch advances) read as zero.
static bool encode_row_tiles(CUtensorMap* tm, const FwdArgs& a, int rows) {
  const cuuint64_t dims[3] = {32, (cuuint64_t)(a.in_avail / 32), (cuuint64_t)a.C};
  const cuuint64_t strides[2] = {128, (cuuint64_t)a.in_stride * 4};
  const cuuint32_t box[3] = {32, (cuuint32_t)rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(a.in), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_tmw6(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s) {
  (void)cfg;
  if (dtype != DD_F32_F32 || !tmw6_accepts(a.in, a.in_stride) || a.hex_desc == nullptr || a.in_avail % 32 != 0 ||
      a.in_avail < a.n_in)
    return cudaErrorInvalidConfiguration;
  CUtensorMap tm;
  if (!encode_row_tiles(&tm, a, kQRows)) return cudaErrorInvalidValue;
  auto kern = a.w ? fwd_tmw6_kernel<true> : fwd_tmw6_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((a.n_dm + kT - 1) / kT), (unsigned)((a.n_out + kBT - 1) / kBT));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  kern<<<grid, kThreads, kSmem, s>>>(tm, a);
  return cudaGetLastError();
}

std::vector<TileConfig> tmw6_menu(dd_dtype dtype) {
  std::vector<TileConfig> v;
  if (dtype != DD_F32_F32) return v;
  v.push_back({Kind::TmW6, kT, kBT, 1, kWS, kThreads, 32, kSmem, 0, "tmw6_f32_d6_t4096"});
  return v;
}

}  // namespace dd
