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
};
