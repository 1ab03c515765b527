// Internal declarations shared by the host API and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dd.h"
#include "nvtx3/nvToolsExt.h"

namespace dd {

// NVTX range over one API call, shown by Nsight tools (no cost without one).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Forward kernel families.  NAIVE is the paper's "generically tuned" layout
// (Section 5: one DM per thread, 1-D blocks, no explicit data reuse); STAGED is
// the 2-D (DM x time) block of Section 2.2 with each channel's input span
// staged in shared memory by bulk copies; U8PK is the uint8 path with packed
// 16-bit integer sums; TMW6 (float) shares each channel's input window among
// 6 DM trials through Tensor Memory; TMW9 (float) shares it among 9 trials
// and copies windows at 4-float granularity.
enum class Kind : int { Naive = 0, Staged = 1, U8Pk = 4, TmW6 = 7, TmW9 = 9 };

struct TileConfig {
  Kind kind;
  int bd;       // DM trials per block
  int bt;       // output samples per block
  int cc;       // channels per pipeline stage
  int stages;   // pipeline depth
  int threads;  // threads per block
  int spl;      // TMW6: samples per lane
  int smem;     // dynamic shared memory bytes (filled per plan)
  int pitch;    // staged row pitch in elements (filled per plan)
  std::string name;
};

// Arguments every forward launcher receives (device pointers).
struct FwdArgs {
  const void* in;
  int64_t in_stride;
  int64_t in_avail;        // elements from `in` to the end of its row (in_stride - the launch's first sample)
  const float* w;
  void* out;
  int64_t out_stride;
  const int32_t* delays;   // [n_dm][C]
  const int32_t* delaysT;  // [C][n_dm_pad], DMs >= n_dm repeat the last trial
  const int4* hex_desc;    // 6-trial group descriptors [ceil(n_dm / 6)][C], or null
  const int4* nine_desc;   // 9-trial group descriptors [ceil(n_dm / 9)][C], or null
  int32_t C;
  int32_t n_dm;
  int32_t n_dm_pad;
  int64_t n_out;
  int64_t n_in;
  int* status;             // device error word
};

// ------------------------------------------------------------- batches
// One beam of a persistent batch launch: its forward arguments, its staged
// row pitch (staged / U8PK configurations), the x extent of the grid its
// plain launch would have, and its first work item.
struct BatchBeam {
  FwdArgs a;
  int pitch;
  int nx;
  int first;
  int pad_;
};
// A persistent launch's work, passed whole as the kernel's parameter (read-only
// constant-bank data, which the compiler may reload at will, where arguments in
// global memory would be reloaded after every barrier wait): beams[0 ..
// n_beams) in the order their items are numbered (longest first), n_items
// tiles in all, and the counter the blocks take items from (zeroed before the
// launch).  Item j of a beam is the plain launch's block (x = j % nx, y = j /
// nx).  TMW9 beams' eight tensor maps each sit in global memory (`maps`,
// [n_beams][8], 64-byte aligned).
constexpr int kBeamsPerLaunch = 64;  // 64 x 128 bytes of beams: 8 KB of parameters
struct BatchWork {
  const void* maps;
  int n_beams;
  int n_items;
  int* counter;
  BatchBeam beams[kBeamsPerLaunch];
};
struct WorkItem {
  int beam, x, y;
};

#ifdef __CUDACC__
// Every thread of the block: take the next item (false when the list is
// exhausted).  item_s is a shared word of the block.
__device__ __forceinline__ bool next_item(const BatchWork& w, int& item_s, WorkItem& it) {
  if (threadIdx.x == 0) item_s = atomicAdd(w.counter, 1);
  __syncthreads();
  const int item = item_s;
  __syncthreads();  // every thread has read item_s before the next item overwrites it
  if (item >= w.n_items) return false;
  int lo = 0, hi = w.n_beams - 1;  // the last beam whose first item <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (w.beams[mid].first <= item) lo = mid;
    else hi = mid - 1;
  }
  const int j = item - w.beams[lo].first, nx = w.beams[lo].nx;
  it.beam = lo;
  it.x = j % nx;
  it.y = j / nx;
  return true;
}

// Every thread of the block: copy beam `k` of the work to `beam_s` (shared
// memory) for a tile that reads its arguments there.  The caller has made
// sure that no thread still reads the previous beam.
__device__ __forceinline__ void copy_beam(const BatchWork& w, int k, BatchBeam& beam_s) {
  static_assert(sizeof(BatchBeam) % 4 == 0 && sizeof(BatchBeam) / 4 <= 64, "one word per thread");
  if (threadIdx.x < sizeof(BatchBeam) / 4)
    reinterpret_cast<int*>(&beam_s)[threadIdx.x] = reinterpret_cast<const int*>(&w.beams[k])[threadIdx.x];
  __syncthreads();
}
#endif

// Select the configuration recorded for this plan in the database named by
// the DD_TUNE_DB environment variable, if there is one (tune.cpp).
void apply_tune_db(dd_plan_s* plan);
// The tuning database key of a plan: device name, geometry and dtype (tune.cpp).
std::string tune_key_of(const dd_plan_s& p);

// TMW6 needs 16-byte aligned input rows of a multiple of 32 floats (128 bytes).
bool tmw6_accepts(const void* in, int64_t in_stride);
// TMW9 needs a 16-byte aligned input whose rows hold every needed sample in
// whole 32-float rows of each of its eight tensor-map views (28 spare floats
// per row are enough); tmw9_min_in_stride gives the smallest such stride.
bool tmw9_accepts(const void* in, int64_t in_stride, int64_t n_in);
int64_t tmw9_min_in_stride(int64_t n_in);

// Forward launch on a given configuration.
cudaError_t launch_forward(const TileConfig& cfg, dd_dtype dtype, const FwdArgs& a, cudaStream_t s);

// Sizes, device tables and configuration menu of a plan whose host delay
// table is filled in (dd_plan.cpp).
dd_status finish_plan(dd_plan_s* p);
void free_plan_device(dd_plan_s* p);
// Indices of a plan's configurations, most promising first (the measured
// preference list, then the rest of the menu, the generic kernels last).
std::vector<int> config_preference_order(const dd_plan_s& p);
// Forward arguments of a plan over output samples [t0, t1) (dd_api.cpp), and
// the configuration a launch with them runs: the plan's choice (or
// cfg_override >= 0), unless the input's layout needs another one.
FwdArgs plan_args(const dd_plan_s* p, const void* in, int64_t in_stride, const float* w, void* out,
                  int64_t out_stride, int64_t t0, int64_t t1);
const TileConfig* resolve_config(const dd_plan_s* p, const FwdArgs& a, int cfg_override);
// Persistent forms for batches (fwd_kernels.cu, fwd_tmw9.cu): does the
// configuration have one, its dynamic shared memory for a staged row pitch,
// its resident blocks per SM at that shared memory and the plain kernel's (0:
// cannot launch), and the launch over a work list with `grid` blocks (at most
// the resident ones, which then take every item in turn).  TMW9 beams need their eight tensor maps in the work's `maps`
// (tmw9_encode_views writes them, tmw9_views_bytes of them per beam).
bool has_persistent(const TileConfig& cfg, dd_dtype dtype);
int persistent_smem(const TileConfig& cfg, dd_dtype dtype, int pitch);
int persistent_blocks_per_sm(const TileConfig& cfg, dd_dtype dtype, int smem);
int plain_blocks_per_sm(const TileConfig& cfg, dd_dtype dtype, int smem);
cudaError_t launch_persistent(const TileConfig& cfg, dd_dtype dtype, const BatchWork& w, int smem, int grid,
                              cudaStream_t s);
size_t tmw9_views_bytes();
bool tmw9_encode_views(const FwdArgs& a, void* out);
// Weight gradient on the TMW9 tiles (fwd_tmw9.cu): the partial sums it
// needs (floats; 0 if the plan or the input layout does not take TMW9), and
// the launch (grad_out [n_dm][g_stride], the partials' scratch, grad_w [C]).
int64_t tmw9_wgrad_partials(const FwdArgs& a);
cudaError_t launch_tmw9_wgrad(const FwdArgs& a, const float* g, int64_t g_stride, float* partial, float* grad_w,
                              cudaStream_t s);
const void* tmw9_persistent_kernel();
const void* tmw9_plain_kernel();
// Validated forward launch (dd_api.cpp); cfg_override < 0 uses the plan's choice.
dd_status forward_device(dd_plan_s* p, const void* in, int64_t in_stride, const float* w, void* out,
                         int64_t out_stride, cudaStream_t stream, int cfg_override);

// Shared-memory limit for one block (opt-in maximum on sm_103a).
constexpr int kMaxSmemPerBlock = 227 * 1024;

// The transposed delay table's rows hold n_dm rounded up to a multiple of
// kDmPad trials (the padding repeats the last trial).  A block that reads the
// delays of trials [i0, i0 + BD) stays inside its row only if BD divides kDmPad.
constexpr int kDmPad = 64;

// TMW6: the largest offset between a 6-trial group's first and last trial
// that its Tensor Memory windows can hold.
constexpr int kW6MaxOff = 31;
// TMW9: the same for a 9-trial group.
constexpr int kW9MaxOff = 31;

// Input row stride (elements) that every forward configuration of a plan
// takes: float rows with TMW9's spare samples, uint8 rows of 128 bytes.
int64_t plan_in_stride(const dd_plan_s& p);
// Device bytes of a stream's two state buffers [C][plan_in_stride] for its
// chunk plan (the plan's geometry with n_out = chunk length).
int64_t stream_buffer_bytes(const dd_plan_s& chunk_plan);

}  // namespace dd

struct dd_plan_s {
  int device = 0;
  int32_t C = 0, n_dm = 0, n_dm_pad = 0;
  int64_t n_out = 0, n_in = 0;
  int32_t max_delay = 0;
  double f_low = 0, chan_bw = 0, t_samp = 0, dm_first = 0, dm_step = 0;
  int32_t dm_index0 = 0;              // trial i of the plan is trial dm_index0 + i of the DM grid
  dd_dtype dtype = DD_F32_F32;
  std::vector<int32_t> delays;        // host copy [n_dm][C]
  int32_t* d_delays = nullptr;        // [n_dm][C]
  int32_t* d_delaysT = nullptr;       // [C][n_dm_pad]
  int4* d_hex_desc = nullptr;         // [ceil(n_dm / 6)][C], float plans whose offsets fit a window
  int4* d_nine_desc = nullptr;        // [ceil(n_dm / 9)][C], likewise for 9-trial groups
  int* d_status = nullptr;            // device error word
  int64_t device_bytes = 0;
  std::vector<dd::TileConfig> configs;
  int selected = 0;
  int fallback = 0;                   // staged configuration for inputs the selected one cannot take
  // host-buffer forward staging (allocated on first dd_forward_host)
  void* h_dev_in = nullptr;
  void* h_dev_out = nullptr;
  float* h_dev_w = nullptr;
  size_t h_in_bytes = 0, h_out_bytes = 0;
  cudaStream_t h_streams[5] = {};     // host-buffer pipeline: copy-in, 2 kernel, 2 copy-out streams
  std::vector<cudaEvent_t> h_events;  // fork, done, then (copied-in, computed) per chunk
  // adjoint: the transposed plan (channels and DM trials swapped, delays
  // max_delay - delay) and its zero-padded copy of grad_out
  dd_plan_s* adj = nullptr;
  float* adj_pad = nullptr;       // [n_dm][adj_pad_stride]
  int64_t adj_pad_stride = 0;
  float* adj_g = nullptr;         // [C][adj_g_stride] unweighted transpose when grad_in is not requested
  int64_t adj_g_stride = 0;
  float* adj_wpart = nullptr;     // per-warp shares of the weight gradient on the TMW9 tiles
  int64_t adj_wpart_floats = 0;
};
