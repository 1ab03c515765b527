// Plans: the delay table of Eq. 1 on the host, its device copies, and the
// per-plan tile configuration menu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "dd_errors.h"
#include "dd_internal.h"

namespace dd {

std::vector<TileConfig> staged_menu(dd_dtype dtype);
std::vector<TileConfig> u8pk_menu(dd_dtype dtype);
std::vector<TileConfig> tmw6_menu(dd_dtype dtype);
std::vector<TileConfig> tmw9_menu(dd_dtype dtype);
int u8pk_smem_for(const TileConfig& cfg, int pitch);
int staged_smem_for(dd_dtype dtype, int stages, int cc, int bd, int pitch);

// Eq. 1 (Section 2): delay in seconds of channel frequency f relative to the
// top of the band f_h is 4150 * DM * (1/f^2 - 1/f_h^2) (MHz); divided by the
// sampling time and rounded half up to a whole number of samples.  Evaluated
// in IEEE double, never in float: float flips entries that lie within 1e-6
// samples of a rounding boundary.
static dd_status compute_delay_table(dd_plan_s& p) {
  const double f_h = p.f_low + (double)(p.C - 1) * p.chan_bw;
  const double inv_fh2 = 1.0 / (f_h * f_h);
  p.delays.assign((size_t)p.n_dm * p.C, 0);
  for (int32_t i = 0; i < p.n_dm; ++i) {
    const double kdm = 4150.0 * (p.dm_first + (double)(p.dm_index0 + i) * p.dm_step);
    for (int32_t c = 0; c < p.C; ++c) {
      const double f = p.f_low + (double)c * p.chan_bw;
      const double samples = kdm * (1.0 / (f * f) - inv_fh2) / p.t_samp;
      const double r = std::floor(samples + 0.5);
      if (!(r >= 0.0) || r > 2147483647.0)
        return set_error(DD_ERR_ARG, "delay of channel %d at DM trial %d does not fit int32 (%.3g samples)", c,
                         i, samples);
      p.delays[(size_t)i * p.C + c] = (int32_t)r;
    }
  }
  return DD_OK;
}

// Largest (delay(c, i + bd - 1) - delay(c, i)) over channels and block starts i
// that are multiples of bd: the widest extra span a block of bd DM trials
// needs beyond its bt samples.  Trials past n_dm repeat the last one.
static int32_t block_spread(const dd_plan_s& p, int bd) {
  int32_t best = 0;
  for (int32_t i0 = 0; i0 < p.n_dm; i0 += bd) {
    const int32_t il = std::min(i0 + bd - 1, p.n_dm - 1);
    for (int32_t c = 0; c < p.C; ++c) {
      const int32_t s = p.delays[(size_t)il * p.C + c] - p.delays[(size_t)i0 * p.C + c];
      best = std::max(best, s);
    }
  }
  return best;
}

// Descriptor of (channel c, group of 6 trials starting at 6g), stored
// group-major ([g][c]: a block reads consecutive entries), for windows
// aligned down to 4 floats: x = delay of the group's first trial; y, z = the
// column of each trial's first sample in the window, (x & 3) + offset, one
// byte each (trials 0..3 in y, 4..5 in z); w = window width in floats,
// (x & 3) + 32 + the largest offset.  Returns the largest offset seen.
static int32_t build_hex_desc(const dd_plan_s& p, std::vector<int4>& desc) {
  const int32_t n_g = (p.n_dm + 5) / 6;
  desc.assign((size_t)p.C * n_g, int4{0, 0, 0, 0});
  int32_t worst = 0;
  for (int32_t c = 0; c < p.C; ++c) {
    for (int32_t g = 0; g < n_g; ++g) {
      const int32_t base = p.delays[(size_t)(6 * g) * p.C + c];
      const int32_t sh = base & 3;
      uint32_t packed[2] = {0, 0};
      int32_t mx = 0;
      for (int j = 0; j < 6; ++j) {
        const int32_t i = std::min(6 * g + j, p.n_dm - 1);
        const int32_t o = p.delays[(size_t)i * p.C + c] - base;
        mx = std::max(mx, o);
        packed[j / 4] |= (uint32_t)std::min(sh + o, 255) << (8 * (j % 4));
      }
      worst = std::max(worst, mx);
      desc[(size_t)g * p.C + c] = int4{base, (int)packed[0], (int)packed[1], sh + 32 + mx};
    }
  }
  return worst;
}

// Descriptor of (channel c, group of 9 trials starting at 9g), group-major
// ([g][c]), for windows that start at the 4-float boundary at or below the
// group's first sample: x = delay of the group's first trial; bytes 0..2 of
// y, z, w = the column of the first sample of trials 0..2, 3..5, 6..8 in the
// window, (x & 3) + offset (the warp reading trials 3p..3p+2 takes word p);
// byte 3 of y = the window's 4-float chunks, ceil(((x & 3) + 32 + largest
// offset) / 4).  Returns the largest offset seen.
static int32_t build_nine_desc(const dd_plan_s& p, std::vector<int4>& desc) {
  const int32_t n_g = (p.n_dm + 8) / 9;
  desc.assign((size_t)p.C * n_g, int4{0, 0, 0, 0});
  int32_t worst = 0;
  for (int32_t c = 0; c < p.C; ++c) {
    for (int32_t g = 0; g < n_g; ++g) {
      const int32_t base = p.delays[(size_t)(9 * g) * p.C + c];
      const int32_t sh = base & 3;
      uint32_t word[3] = {0, 0, 0};
      int32_t mx = 0;
      for (int j = 0; j < 9; ++j) {
        const int32_t i = std::min(9 * g + j, p.n_dm - 1);
        const int32_t o = p.delays[(size_t)i * p.C + c] - base;
        mx = std::max(mx, o);
        word[j / 3] |= (uint32_t)std::min(sh + o, 255) << (8 * (j % 3));
      }
      worst = std::max(worst, mx);
      const uint32_t nch = (uint32_t)std::min((sh + 32 + mx + 3) / 4, 255);
      desc[(size_t)g * p.C + c] = int4{base, (int)(word[0] | nch << 24), (int)word[1], (int)word[2]};
    }
  }
  return worst;
}

int32_t block_spread_of(const dd_plan_s& p, int bd) { return block_spread(p, bd); }

// Device memory of a plan's tables, from its host delay table alone: the
// table [n_dm][C], its transposed padded copy [C][n_dm_pad], the status word,
// and the 6- and 9-trial window descriptors where a group's offsets fit the
// Tensor-Memory windows (float plans).  finish_plan allocates exactly these;
// the footprint queries report the same numbers without allocating.
struct TableSizes {
  size_t delays = 0, delays_t = 0, status = sizeof(int), hex = 0, nine = 0;
  int64_t total() const { return (int64_t)(delays + delays_t + status + hex + nine); }
};
static TableSizes table_sizes(const dd_plan_s& p) {
  TableSizes t;
  const int64_t n_dm_pad = (p.n_dm + kDmPad - 1) / kDmPad * kDmPad;
  t.delays = (size_t)p.n_dm * p.C * 4;
  t.delays_t = (size_t)p.C * n_dm_pad * 4;
  if (p.dtype == DD_F32_F32) {
    // a group's largest offset is its last trial's delay less its first's
    if (block_spread(p, 6) <= kW6MaxOff) t.hex = (size_t)p.C * ((p.n_dm + 5) / 6) * sizeof(int4);
    if (block_spread(p, 9) <= kW9MaxOff) t.nine = (size_t)p.C * ((p.n_dm + 8) / 9) * sizeof(int4);
  }
  return t;
}

int64_t plan_in_stride(const dd_plan_s& p) {
  if (p.dtype == DD_U8_I32) return (p.n_in + 127) / 128 * 128;
  return tmw9_min_in_stride(p.n_in);
}

int64_t stream_buffer_bytes(const dd_plan_s& chunk_plan) {
  const int64_t elem = chunk_plan.dtype == DD_U8_I32 ? 1 : 4;
  return 2 * (int64_t)chunk_plan.C * plan_in_stride(chunk_plan) * elem;
}

void free_plan_device(dd_plan_s* p) {
  cudaFree(p->d_delays);
  cudaFree(p->d_delaysT);
  cudaFree(p->d_hex_desc);
  cudaFree(p->d_nine_desc);
  cudaFree(p->d_status);
  cudaFree(p->h_dev_in);
  cudaFree(p->h_dev_out);
  cudaFree(p->h_dev_w);
  for (int k = 0; k < 5; ++k)
    if (p->h_streams[k]) cudaStreamDestroy(p->h_streams[k]);
  for (cudaEvent_t ev : p->h_events) cudaEventDestroy(ev);
  p->h_events.clear();
  cudaFree(p->adj_pad);
  cudaFree(p->adj_g);
  cudaFree(p->adj_wpart);
  if (p->adj) {
    free_plan_device(p->adj);
    delete p->adj;
    p->adj = nullptr;
  }
  p->d_delays = p->d_delaysT = nullptr;
  p->d_hex_desc = nullptr;
  p->d_nine_desc = nullptr;
  p->d_status = nullptr;
  p->h_dev_in = p->h_dev_out = nullptr;
  p->h_dev_w = nullptr;
  for (int k = 0; k < 5; ++k) p->h_streams[k] = nullptr;
  p->adj_pad = p->adj_g = nullptr;
  p->adj_wpart = nullptr;
  p->adj_wpart_floats = 0;
}

// Default configuration: the first valid entry of a preference list, in
// the order measured on the Table 2 setups (Apertif float: TMW9, TMW6 4.07 ms,
// staged d8/t1024 4.94 ms; LOFAR float: staged d8/t1024 3.16 ms, d32/t384
// 3.12 ms; Apertif uint8: U8PK 4 trials/warp c24 2.10 ms); dd_tune replaces it with a
// measured choice.  TMW6 is offered only where a 6-trial group's offsets fit
// its windows (Apertif, not LOFAR).
static const char* const kPrefsF32[] = {"tmw9_f32_d9_t4096",     "tmw6_f32_d6_t4096",     "staged_d8_t1024_c4_s3",
                                        "staged_d16_t512_c8_s3",
                                        "staged_d32_t512_c8_s2", "staged_d32_t384_c4_s3", "staged_d16_t256_c8_s3",
                                        "naive_t256"};
static const char* const kPrefsU8[] = {"u8pk_w8x1_d4_c24_st3", "u8pk_w8x1_d4_c16_st3", "u8pk_w8x1_d2_c32_st3",
                                       "u8pk_w8x1_d2_c16_st4", "staged_d16_t512_c8_s3", "staged_d8_t1024_c4_s3",
                                       "naive_t256"};

// uint8 beams with fewer than 1024 channels: two trials per warp (measured
// on 32- and 256-channel beams of both grids: up to 2.5x faster than four)
static const char* const kPrefsU8Narrow[] = {"u8pk_w8x1_d2_c32_st3", "u8pk_w8x1_d2_c16_st4", "u8pk_w8x1_d4_c24_st3",
                                             "u8pk_w8x1_d4_c16_st3", "staged_d16_t512_c8_s3",
                                             "staged_d8_t1024_c4_s3", "naive_t256"};

static void pref_list(const dd_plan_s& p, const char* const** prefs, size_t* n) {
  if (p.dtype != DD_U8_I32) {
    *prefs = kPrefsF32;
    *n = sizeof(kPrefsF32) / sizeof(kPrefsF32[0]);
  } else if (p.C < 1024) {
    *prefs = kPrefsU8Narrow;
    *n = sizeof(kPrefsU8Narrow) / sizeof(kPrefsU8Narrow[0]);
  } else {
    *prefs = kPrefsU8;
    *n = sizeof(kPrefsU8) / sizeof(kPrefsU8[0]);
  }
}

static int preferred(const dd_plan_s& p, bool staged_only) {
  const char* const* prefs = nullptr;
  size_t n = 0;
  pref_list(p, &prefs, &n);
  for (size_t k = 0; k < n; ++k)
    for (size_t j = 0; j < p.configs.size(); ++j)
      if (p.configs[j].name == prefs[k] && (!staged_only || p.configs[j].kind == Kind::Staged)) return (int)j;
  for (size_t j = 0; j < p.configs.size(); ++j)
    if (!staged_only || p.configs[j].kind == Kind::Staged) return (int)j;
  return 0;
}
static int default_config(const dd_plan_s& p) { return preferred(p, false); }

std::vector<int> config_preference_order(const dd_plan_s& p) {
  // the preference list first (its measured order), then the rest of the
  // menu, generic kernels last
  const char* const* prefs = nullptr;
  size_t n = 0;
  pref_list(p, &prefs, &n);
  std::vector<int> order;
  std::vector<char> seen(p.configs.size(), 0);
  auto take = [&](size_t j) {
    if (!seen[j]) {
      seen[j] = 1;
      order.push_back((int)j);
    }
  };
  for (size_t k = 0; k < n; ++k)
    for (size_t j = 0; j < p.configs.size(); ++j)
      if (p.configs[j].name == prefs[k] && p.configs[j].kind != Kind::Naive) take(j);
  for (size_t j = 0; j < p.configs.size(); ++j)
    if (p.configs[j].kind != Kind::Naive) take(j);
  for (size_t j = 0; j < p.configs.size(); ++j) take(j);
  return order;
}
// The configuration used when the selected one cannot take an input's
// layout (TMW6 needs 128-byte rows): the preferred shared-memory kernel.
static int fallback_config(const dd_plan_s& p) { return preferred(p, true); }

// Everything a plan derives from its delay table (p->delays [n_dm][C], rows
// non-decreasing along the trial index for every channel): sizes, device
// copies of the table and descriptors, and the configuration menu.
dd_status finish_plan(dd_plan_s* p) {
  p->max_delay = *std::max_element(p->delays.begin(), p->delays.end());
  p->n_in = p->n_out + p->max_delay;
  p->n_dm_pad = (p->n_dm + kDmPad - 1) / kDmPad * kDmPad;

  if (cudaGetDevice(&p->device) != cudaSuccess) return set_cuda_error("dd_plan: cudaGetDevice");
  // transposed, padded copy: [C][n_dm_pad], trials past n_dm repeat the last
  std::vector<int32_t> dT((size_t)p->C * p->n_dm_pad);
  for (int32_t c = 0; c < p->C; ++c)
    for (int32_t i = 0; i < p->n_dm_pad; ++i)
      dT[(size_t)c * p->n_dm_pad + i] = p->delays[(size_t)std::min(i, p->n_dm - 1) * p->C + c];
  const TableSizes sizes = table_sizes(*p);
  const size_t bytes_d = sizes.delays, bytes_dT = sizes.delays_t;
  cudaError_t e = cudaMalloc(&p->d_delays, bytes_d);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_delaysT, bytes_dT);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(p->d_delays, p->delays.data(), bytes_d, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_delaysT, dT.data(), bytes_dT, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    free_plan_device(p);
    return e == cudaErrorMemoryAllocation ? set_error(DD_ERR_NOMEM, "dd_plan: device allocation failed")
                                          : set_cuda_error("dd_plan: upload", e);
  }
  p->device_bytes = (int64_t)(bytes_d + bytes_dT + sizeof(int));
  // 6-trial descriptors, only where the windows fit (float plans, offsets <= 31)
  bool hex_ok = false;
  if (sizes.hex > 0) {
    std::vector<int4> desc6;
    if (build_hex_desc(*p, desc6) <= kW6MaxOff) {
      const size_t bytes6 = desc6.size() * sizeof(int4);
      e = cudaMalloc(&p->d_hex_desc, bytes6);
      if (e == cudaSuccess) e = cudaMemcpy(p->d_hex_desc, desc6.data(), bytes6, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        free_plan_device(p);
        return e == cudaErrorMemoryAllocation ? set_error(DD_ERR_NOMEM, "dd_plan: device allocation failed")
                                              : set_cuda_error("dd_plan: upload", e);
      }
      p->device_bytes += (int64_t)bytes6;
      hex_ok = true;
    }
  }
  bool nine_ok = false;
  if (sizes.nine > 0) {
    std::vector<int4> desc9;
    if (build_nine_desc(*p, desc9) <= kW9MaxOff) {
      const size_t bytes9 = desc9.size() * sizeof(int4);
      e = cudaMalloc(&p->d_nine_desc, bytes9);
      if (e == cudaSuccess) e = cudaMemcpy(p->d_nine_desc, desc9.data(), bytes9, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        free_plan_device(p);
        return e == cudaErrorMemoryAllocation ? set_error(DD_ERR_NOMEM, "dd_plan: device allocation failed")
                                              : set_cuda_error("dd_plan: upload", e);
      }
      p->device_bytes += (int64_t)bytes9;
      nine_ok = true;
    }
  }
  // configuration menu, filtered by what this geometry allows
  const int V = p->dtype == DD_U8_I32 ? 16 : 4;
  for (TileConfig cfg : staged_menu(p->dtype)) {
    if (cfg.kind == Kind::Staged) {
      const int64_t spread = block_spread(*p, cfg.bd);
      const int64_t pitch = (cfg.bt + spread + 2 * V + V - 1) / V * V;
      if (pitch > (int64_t)1 << 20) continue;
      cfg.pitch = (int)pitch;
      cfg.smem = staged_smem_for(p->dtype, cfg.stages, cfg.cc, cfg.bd, cfg.pitch);
      if (cfg.smem > kMaxSmemPerBlock) continue;
      if ((p->n_dm + cfg.bd - 1) / cfg.bd > 65535) continue;
    }
    p->configs.push_back(cfg);
  }
  for (TileConfig cfg : u8pk_menu(p->dtype)) {
    const int64_t spread = block_spread(*p, cfg.bd);
    // + 32: a lane reads 32 bytes from a word-aligned start at or before its first sample
    const int64_t pitch = (cfg.bt + spread + 2 * V + 32 + V - 1) / V * V;
    if (pitch > (int64_t)1 << 20) continue;
    cfg.pitch = (int)pitch;
    cfg.smem = u8pk_smem_for(cfg, cfg.pitch);
    if (cfg.smem > kMaxSmemPerBlock) continue;
    if ((p->n_dm + cfg.bd - 1) / cfg.bd > 65535) continue;
    p->configs.push_back(cfg);
  }
  if (hex_ok) {
    for (TileConfig cfg : tmw6_menu(p->dtype)) {
      if ((p->n_out + cfg.bt - 1) / cfg.bt > 65535) continue;  // time tiles are the grid's y
      p->configs.push_back(cfg);
    }
  }
  if (nine_ok) {
    for (TileConfig cfg : tmw9_menu(p->dtype)) {
      if ((p->n_out + cfg.bt - 1) / cfg.bt > 65535) continue;
      p->configs.push_back(cfg);
    }
  }
  p->selected = default_config(*p);
  p->fallback = fallback_config(*p);
  return DD_OK;
}

}  // namespace dd

using namespace dd;

static dd_status check_plan_args(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                                 double dm_first, double dm_step, int32_t n_dm) {
  if (channels <= 0) return set_error(DD_ERR_ARG, "channels must be > 0 (got %d)", channels);
  if (!(f_low_mhz > 0.0) || !std::isfinite(f_low_mhz)) return set_error(DD_ERR_ARG, "f_low must be > 0 MHz");
  if (!(chan_bw_mhz > 0.0) || !std::isfinite(chan_bw_mhz)) return set_error(DD_ERR_ARG, "chan_bw must be > 0 MHz");
  if (!(t_samp_s > 0.0) || !std::isfinite(t_samp_s)) return set_error(DD_ERR_ARG, "t_samp must be > 0 s");
  if (!(dm_first >= 0.0) || !std::isfinite(dm_first)) return set_error(DD_ERR_ARG, "dm_first must be >= 0");
  if (!(dm_step >= 0.0) || !std::isfinite(dm_step)) return set_error(DD_ERR_ARG, "dm_step must be >= 0");
  if (n_dm <= 0) return set_error(DD_ERR_ARG, "n_dm must be > 0 (got %d)", n_dm);
  if ((int64_t)channels * n_dm > (int64_t)1 << 31)
    return set_error(DD_ERR_ARG, "delay table of %lld entries is too large", (long long)channels * n_dm);
  return DD_OK;
}

extern "C" dd_status dd_delay_table(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                                    double dm_first, double dm_step, int32_t n_dm, int32_t* host_out) {
  return dd_delay_table_dm_range(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, 0, n_dm, host_out);
}

extern "C" dd_status dd_delay_table_dm_range(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                                             double dm_first, double dm_step, int32_t dm_index0, int32_t n_dm,
                                             int32_t* host_out) {
  clear_error();
  if (!host_out) return set_error(DD_ERR_ARG, "dd_delay_table: host_out is NULL");
  dd_status st = check_plan_args(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm);
  if (st != DD_OK) return st;
  if (dm_index0 < 0 || (int64_t)dm_index0 + n_dm > 2147483647LL)
    return set_error(DD_ERR_ARG, "dd_delay_table: first trial index %d out of range", dm_index0);
  dd_plan_s p;
  p.C = channels;
  p.n_dm = n_dm;
  p.f_low = f_low_mhz;
  p.chan_bw = chan_bw_mhz;
  p.t_samp = t_samp_s;
  p.dm_first = dm_first;
  p.dm_step = dm_step;
  p.dm_index0 = dm_index0;
  st = compute_delay_table(p);
  if (st != DD_OK) return st;
  std::memcpy(host_out, p.delays.data(), p.delays.size() * sizeof(int32_t));
  return DD_OK;
}

extern "C" dd_status dd_plan(dd_plan_t* out, int32_t channels, double f_low_mhz, double chan_bw_mhz,
                             double t_samp_s, double dm_first, double dm_step, int32_t n_dm, int64_t n_out,
                             dd_dtype dtype) {
  return dd_plan_dm_range(out, channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, 0, n_dm, n_out, dtype);
}

extern "C" dd_status dd_plan_dm_range(dd_plan_t* out, int32_t channels, double f_low_mhz, double chan_bw_mhz,
                                      double t_samp_s, double dm_first, double dm_step, int32_t dm_index0,
                                      int32_t n_dm, int64_t n_out, dd_dtype dtype) {
  clear_error();
  if (!out) return set_error(DD_ERR_ARG, "dd_plan: out is NULL");
  dd_status chk = check_plan_args(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm);
  if (chk != DD_OK) return chk;
  if (dm_index0 < 0 || (int64_t)dm_index0 + n_dm > 2147483647LL)
    return set_error(DD_ERR_ARG, "dd_plan_dm_range: first trial index %d out of range", dm_index0);
  if (n_out <= 0) return set_error(DD_ERR_ARG, "dd_plan: n_out must be > 0");
  if (dtype != DD_U8_I32 && dtype != DD_F32_F32) return set_error(DD_ERR_ARG, "dd_plan: unknown dtype %d", (int)dtype);
  if (dtype == DD_U8_I32 && (int64_t)channels * 255 > 2147483647LL)
    return set_error(DD_ERR_ARG, "dd_plan: %d channels of uint8 overflow int32 sums", channels);

  dd_plan_s* p = new (std::nothrow) dd_plan_s();
  if (!p) return set_error(DD_ERR_NOMEM, "dd_plan: host allocation failed");
  p->C = channels;
  p->n_dm = n_dm;
  p->n_out = n_out;
  p->f_low = f_low_mhz;
  p->chan_bw = chan_bw_mhz;
  p->t_samp = t_samp_s;
  p->dm_first = dm_first;
  p->dm_step = dm_step;
  p->dm_index0 = dm_index0;
  p->dtype = dtype;
  dd_status st = compute_delay_table(*p);
  if (st != DD_OK) {
    delete p;
    return st;
  }
  st = finish_plan(p);
  if (st != DD_OK) {
    delete p;
    return st;
  }
  apply_tune_db(p);
  *out = p;
  return DD_OK;
}

// A host-only plan of the given geometry with its delay table (no device
// memory), for the footprint queries.
static dd_status host_plan(dd_plan_s& p, int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                           double dm_first, double dm_step, int32_t n_dm, int64_t n_out, dd_dtype dtype) {
  dd_status st = check_plan_args(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm);
  if (st != DD_OK) return st;
  if (dtype != DD_U8_I32 && dtype != DD_F32_F32) return set_error(DD_ERR_ARG, "unknown dtype %d", (int)dtype);
  p.C = channels;
  p.n_dm = n_dm;
  p.n_out = n_out;
  p.f_low = f_low_mhz;
  p.chan_bw = chan_bw_mhz;
  p.t_samp = t_samp_s;
  p.dm_first = dm_first;
  p.dm_step = dm_step;
  p.dtype = dtype;
  st = compute_delay_table(p);
  if (st != DD_OK) return st;
  p.max_delay = *std::max_element(p.delays.begin(), p.delays.end());
  p.n_in = p.n_out + p.max_delay;
  return DD_OK;
}

extern "C" dd_status dd_plan_footprint(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                                       double dm_first, double dm_step, int32_t n_dm, dd_dtype dtype,
                                       int64_t* device_bytes) {
  clear_error();
  if (!device_bytes) return set_error(DD_ERR_ARG, "dd_plan_footprint: device_bytes is NULL");
  dd_plan_s p;
  dd_status st = host_plan(p, channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm, 1, dtype);
  if (st != DD_OK) return st;
  *device_bytes = table_sizes(p).total();
  return DD_OK;
}

extern "C" dd_status dd_stream_footprint(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                                         double dm_first, double dm_step, int32_t n_dm, int64_t chunk_len,
                                         dd_dtype dtype, int64_t* device_bytes) {
  clear_error();
  if (!device_bytes) return set_error(DD_ERR_ARG, "dd_stream_footprint: device_bytes is NULL");
  if (chunk_len <= 0) return set_error(DD_ERR_ARG, "dd_stream_footprint: chunk_len must be > 0");
  dd_plan_s p;  // the stream's own plan: the same geometry, n_out = chunk_len
  dd_status st = host_plan(p, channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm, chunk_len, dtype);
  if (st != DD_OK) return st;
  *device_bytes = table_sizes(p).total() + stream_buffer_bytes(p);
  return DD_OK;
}

extern "C" dd_status dd_plan_destroy(dd_plan_t plan) {
  clear_error();
  if (!plan) return DD_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  free_plan_device(plan);
  if (prev >= 0 && prev != plan->device) cudaSetDevice(prev);
  delete plan;
  return DD_OK;
}

extern "C" dd_status dd_plan_info(dd_plan_t plan, int64_t* n_in, int32_t* max_delay, int64_t* device_bytes) {
  clear_error();
  if (!plan) return set_error(DD_ERR_ARG, "dd_plan_info: plan is NULL");
  if (n_in) *n_in = plan->n_in;
  if (max_delay) *max_delay = plan->max_delay;
  if (device_bytes) *device_bytes = plan->device_bytes;
  return DD_OK;
}

extern "C" dd_status dd_plan_in_stride(dd_plan_t plan, int64_t* in_row_stride) {
  clear_error();
  if (!plan || !in_row_stride) return set_error(DD_ERR_ARG, "dd_plan_in_stride: NULL argument");
  *in_row_stride = plan_in_stride(*plan);
  return DD_OK;
}

extern "C" dd_status dd_plan_delays(dd_plan_t plan, int32_t* host_out) {
  clear_error();
  if (!plan || !host_out) return set_error(DD_ERR_ARG, "dd_plan_delays: NULL argument");
  std::memcpy(host_out, plan->delays.data(), plan->delays.size() * sizeof(int32_t));
  return DD_OK;
}

extern "C" dd_status dd_plan_num_configs(dd_plan_t plan, int32_t* n) {
  clear_error();
  if (!plan || !n) return set_error(DD_ERR_ARG, "dd_plan_num_configs: NULL argument");
  *n = (int32_t)plan->configs.size();
  return DD_OK;
}

extern "C" const char* dd_plan_config_name(dd_plan_t plan, int32_t k) {
  if (!plan || k < 0 || k >= (int32_t)plan->configs.size()) return nullptr;
  return plan->configs[k].name.c_str();
}

extern "C" dd_status dd_plan_select_config(dd_plan_t plan, int32_t k) {
  clear_error();
  if (!plan) return set_error(DD_ERR_ARG, "dd_plan_select_config: plan is NULL");
  if (k < 0 || k >= (int32_t)plan->configs.size())
    return set_error(DD_ERR_ARG, "dd_plan_select_config: config %d out of range [0, %zu)", k, plan->configs.size());
  plan->selected = k;
  return DD_OK;
}

extern "C" dd_status dd_plan_selected_config(dd_plan_t plan, int32_t* k) {
  clear_error();
  if (!plan || !k) return set_error(DD_ERR_ARG, "dd_plan_selected_config: NULL argument");
  *k = plan->selected;
  return DD_OK;
}

extern "C" dd_status dd_plan_device_status(dd_plan_t plan, int32_t* code) {
  clear_error();
  if (!plan || !code) return set_error(DD_ERR_ARG, "dd_plan_device_status: NULL argument");
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_cuda_error("dd_plan_device_status", e);
  *code = v;
  if (v != 0) {
    cudaMemset(plan->d_status, 0, sizeof(int));
    return set_error(DD_ERR_STATE, "a kernel of this plan reported device error %d (1 = bounded wait expired)", v);
  }
  return DD_OK;
}
