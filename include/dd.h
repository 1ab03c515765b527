/*
 * libdd: brute-force incoherent dedispersion on NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Every entry point takes plain host/device pointers and sizes; no C++
 * or framework type crosses this boundary.  The method is the one of
 * Sclocco et al., "Real-Time Dedispersion for Fast Radio Transient Surveys,
 * using Auto Tuning on Many-Core Accelerators":
 *
 *   out[dm][t] = sum over c of w[c] * in[c][t + delay(c, dm)]      (Algorithm 1)
 *   delay(c, dm) = round(4150 * DM * (1/f_c^2 - 1/f_h^2) / t_samp)   (Eq. 1)
 *
 * Conventions shared by every call:
 *  - Frequencies in MHz, times in seconds, DM in pc cm^-3.  Channel c has
 *    frequency f_low + c * chan_bw; channel 0 is the lowest, f_h is channel
 *    C-1 (its delay is 0).  DM trial i is dm_first + i * dm_step.
 *  - Delays are whole samples, Eq. 1 evaluated in IEEE double and rounded half
 *    up (the paper does not say how to round).
 *  - The input of one beam is a row-major [channels][in_row_stride] matrix
 *    whose first n_in = n_out + max_delay samples per row are read (Section 2.1:
 *    the t samples needed to produce s output samples).  The output is a
 *    row-major [n_dm][out_row_stride] matrix; the first n_out entries of each
 *    row are written.  Strides are in elements, not bytes.
 *  - Data buffers (input, output, weights, gradients) are owned by the caller.
 *    Plans, batches and stream states are owned by the library and freed by
 *    their destroy call.
 *  - Calls that take a `stream` (a cudaStream_t, NULL = legacy default stream)
 *    are asynchronous: they enqueue work and return.  Pointers passed to them
 *    must be device (or managed) memory of the plan's device unless the call
 *    says "host".  Errors are returned as a status, never by aborting; a
 *    human-readable detail for the last failing call on the calling thread is
 *    available from dd_last_error().
 *  - A plan is bound to the CUDA device that was current when it was made.
 */
#ifndef LIBDD_DD_H
#define LIBDD_DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_plan_s* dd_plan_t;
typedef struct dd_batch_s* dd_batch_t;
typedef struct dd_stream_s* dd_stream_t;

typedef enum {
  DD_OK = 0,
  DD_ERR_ARG = 1,          /* invalid argument: null pointer, non-positive size, bad value */
  DD_ERR_SHAPE = 2,        /* a stride or length too small for the plan */
  DD_ERR_ALIGN = 3,        /* pointer or stride alignment the call requires is not met */
  DD_ERR_NOMEM = 4,        /* a device or host allocation failed */
  DD_ERR_CUDA = 5,         /* a CUDA runtime call failed (detail in dd_last_error) */
  DD_ERR_UNSUPPORTED = 6,  /* combination not supported (e.g. weights on the uint8 path) */
  DD_ERR_BUDGET = 7,       /* request exceeds a memory budget */
  DD_ERR_STATE = 8         /* object in the wrong state for the call */
} dd_status;

typedef enum {
  DD_U8_I32 = 0,   /* uint8 samples, int32 sums, unit weights only: bit-exact */
  DD_F32_F32 = 1   /* float32 samples and weights, float32 sums */
} dd_dtype;

/* ------------------------------------------------------------------ plans */

/*
 * Build a dedispersion plan: computes the delay table of Eq. 1 (Section 2)
 * for n_dm trials x `channels` channels on the host in double precision,
 * rounds it half up to whole samples, and uploads it with the tile
 * descriptors the kernels use to the current device.  Section 2.1: the
 * delays are computed once, in advance, and do not add to the O(d*s*c) cost.
 *
 * channels > 0, f_low_mhz > 0, chan_bw_mhz > 0, t_samp_s > 0, dm_first >= 0,
 * dm_step >= 0, n_dm > 0, n_out > 0.  The largest delay must fit in int32 and
 * the output sums must fit their type (uint8: channels * 255 < 2^31).
 * Returns DD_ERR_ARG on bad values, DD_ERR_NOMEM / DD_ERR_CUDA on device
 * failures.  *out is set only on DD_OK.
 */
dd_status dd_plan(dd_plan_t* out, int32_t channels, double f_low_mhz, double chan_bw_mhz,
                  double t_samp_s, double dm_first, double dm_step, int32_t n_dm,
                  int64_t n_out, dd_dtype dtype);

/*
 * A plan over DM trials [dm_index0, dm_index0 + n_dm) of the grid
 * DM_i = dm_first + i * dm_step: trial j of the plan has DM_(dm_index0 + j),
 * computed exactly as dd_plan computes it, so its delay rows and outputs equal
 * rows dm_index0 .. dm_index0 + n_dm - 1 of the full plan's bit for bit.
 * Beams are split across GPUs this way (Section 2: every DM trial is an
 * independent sum): each GPU reads the whole input and writes its own rows;
 * nothing is reduced.  dm_index0 >= 0 and dm_index0 + n_dm < 2^31; otherwise
 * as dd_plan (dd_plan is dm_index0 = 0).
 */
dd_status dd_plan_dm_range(dd_plan_t* out, int32_t channels, double f_low_mhz, double chan_bw_mhz,
                           double t_samp_s, double dm_first, double dm_step, int32_t dm_index0, int32_t n_dm,
                           int64_t n_out, dd_dtype dtype);

/*
 * Host-only: the delay table of Eq. 1 exactly as dd_plan computes it, written
 * to `host_out` ([n_dm][channels] int32, row-major) without touching a GPU.
 * Same argument rules and errors as dd_plan (DD_ERR_ARG).
 */
dd_status dd_delay_table(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                         double dm_first, double dm_step, int32_t n_dm, int32_t* host_out);

/* Host-only: the delay rows of trials [dm_index0, dm_index0 + n_dm) exactly
 * as dd_plan_dm_range computes them (rows dm_index0 .. of dd_delay_table's
 * full table).  Argument rules and errors as dd_plan_dm_range. */
dd_status dd_delay_table_dm_range(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                                  double dm_first, double dm_step, int32_t dm_index0, int32_t n_dm,
                                  int32_t* host_out);

/* Free a plan and its device memory.  NULL is accepted.  The caller must not
 * destroy a plan while work enqueued with it may still run. */
dd_status dd_plan_destroy(dd_plan_t plan);

/*
 * Sizes derived by the plan (any output pointer may be NULL):
 *   n_in         input samples per channel row that are read, n_out + max_delay;
 *   max_delay    the largest delay in samples (lowest channel, last DM trial);
 *   device_bytes device memory the plan holds (delay table + descriptors).
 */
dd_status dd_plan_info(dd_plan_t plan, int64_t* n_in, int32_t* max_delay, int64_t* device_bytes);

/*
 * The input row stride (elements, >= n_in) that every forward configuration
 * of the plan takes at full speed: for float32, a multiple of 32 floats with
 * at least 28 spare floats after the n_in samples read (the 9-trial Tensor
 * Memory kernel loads 4-float-aligned 128-byte rows that may reach past
 * n_in; the spare floats are read, never used); for uint8, n_in rounded up to
 * 128 bytes.  Other strides >= n_in are accepted and run the fastest
 * configuration that takes them.  Section 2.1: n_in = n_out + max_delay
 * samples per channel.
 */
dd_status dd_plan_in_stride(dd_plan_t plan, int64_t* in_row_stride);

/*
 * Host-only sizing (no device memory is touched): the device bytes that
 * dd_plan of this geometry would hold (dd_plan_info's device_bytes of the
 * plan it makes: the delay table of Eq. 1, its transposed copy, the status
 * word and the window descriptors; n_out does not change it).  Arguments and
 * errors as dd_plan.  For admission control, e.g. a serving loop that keeps
 * beams within an HBM budget.
 */
dd_status dd_plan_footprint(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                            double dm_first, double dm_step, int32_t n_dm, dd_dtype dtype, int64_t* device_bytes);

/* Copy the plan's delay table (Eq. 1, in samples) to host memory `host_out`,
 * row-major [n_dm][channels] int32.  For checking the plan against Eq. 1. */
dd_status dd_plan_delays(dd_plan_t plan, int32_t* host_out);

/*
 * Kernel selection.  A plan carries the tile configuration the forward call
 * launches (the tunable parameters of Section 2.2: work per thread in DM and
 * time, threads per block in DM and time, staging in shared memory or not).
 * dd_plan_num_configs gives how many configurations are valid for the plan;
 * dd_plan_config_name(plan, k) returns a static description of config k
 * (NULL if out of range); dd_plan_select_config makes config k the one
 * dd_forward uses; dd_plan_selected_config reports it.  A new plan starts at
 * a built-in heuristic choice.
 */
dd_status dd_plan_num_configs(dd_plan_t plan, int32_t* n);
const char* dd_plan_config_name(dd_plan_t plan, int32_t k);
dd_status dd_plan_select_config(dd_plan_t plan, int32_t k);
dd_status dd_plan_selected_config(dd_plan_t plan, int32_t* k);

/*
 * Failure detection.  Every wait inside the library's kernels is bounded
 * (about one second); a wait that expires makes the kernel record a nonzero
 * code in the plan's device status word and return early instead of hanging.
 * This call waits for the device, reads that word into *code and clears it:
 * DD_OK if it was 0, DD_ERR_STATE otherwise (1 = a bounded wait expired).
 */
dd_status dd_plan_device_status(dd_plan_t plan, int32_t* code);

/*
 * Self-check of that path (not in the paper): launches on `stream` a one-warp
 * kernel that waits, with a limit of `limit_cycles` SM clock cycles (1 ..
 * 2e9), on an mbarrier phase nothing completes.  The wait expires, the
 * kernel records code 1 in the plan's status word and returns, and the
 * context stays usable; dd_plan_device_status then reports it.  Errors:
 * DD_ERR_ARG (NULL plan, limit out of range), DD_ERR_CUDA (launch failure).
 */
dd_status dd_check_wait_timeout(dd_plan_t plan, int64_t limit_cycles, void* stream);

/* ---------------------------------------------------------------- forward */

/*
 * Algorithm 1 (Section 2.1) on one beam:
 *   out[i][t] = sum_c w[c] * in[c][t + delay(c, i)],  0 <= i < n_dm, 0 <= t < n_out.
 *
 * in   device, [channels][in_row_stride] of uint8 (DD_U8_I32) or float
 *      (DD_F32_F32); in_row_stride >= n_in.
 * w    device float[channels] or NULL (unit weights).  Must be NULL for
 *      DD_U8_I32 (DD_ERR_UNSUPPORTED otherwise).
 * out  device, [n_dm][out_row_stride] of int32 (DD_U8_I32) or float;
 *      out_row_stride >= n_out.  Overwritten; `in` and `out` must not overlap.
 * The staged kernels need `in` 16-byte aligned and in_row_stride * elem a
 * multiple of 16 bytes; inputs that are not get a plain-load kernel instead
 * (same result).  Errors: DD_ERR_ARG (null plan/in/out), DD_ERR_SHAPE (a
 * stride too small), DD_ERR_UNSUPPORTED, DD_ERR_CUDA (launch failure).
 */
dd_status dd_forward(dd_plan_t plan, const void* in, int64_t in_row_stride, const float* w,
                     void* out, int64_t out_row_stride, void* stream);

/*
 * dd_forward on HOST buffers: copies `host_in` (and `host_w`) to device
 * buffers the plan owns, runs the forward kernel and copies the result back
 * to `host_out`, then waits for `stream`.  Outputs longer than 12288 samples
 * run in three time chunks (4096 samples, the middle, the last partial 4096)
 * as a pipeline on streams the plan owns (one for the copies of the input
 * columns chunk k adds, two each for the kernels and the copies out,
 * alternating between chunks), forked from and joined back into `stream`, so
 * the copies overlap the kernels; the result is bit-identical to one
 * dd_forward.  Layouts as for dd_forward.
 * Page-locked host memory gives full copy bandwidth (and is needed for the
 * copies to overlap).  The plan's staging buffers, streams and events are
 * created on first use and kept until the plan is destroyed (DD_ERR_NOMEM if
 * they cannot be).  Not safe to call concurrently on the same plan.
 */
dd_status dd_forward_host(dd_plan_t plan, const void* host_in, int64_t in_row_stride,
                          const float* host_w, void* host_out, int64_t out_row_stride,
                          void* stream);

/* ---------------------------------------------------------------- adjoint */

/*
 * Transpose and weight gradient of the weighted Algorithm 1 (not in the
 * paper; float32 plans only):
 *   grad_in[c][u] = w[c] * sum over i with 0 <= u - delay(c,i) < n_out of
 *                   grad_out[i][u - delay(c,i)]          for 0 <= u < n_in
 *   grad_w[c]     = sum_i sum_t grad_out[i][t] * in[c][t + delay(c,i)]
 *
 * grad_out device float [n_dm][go_row_stride], go_row_stride >= n_out.
 * w        device float[channels] or NULL (unit weights).
 * grad_in  device float [channels][gi_row_stride], gi_row_stride >= n_in, or
 *          NULL to skip; its first n_in entries per row are overwritten.
 * in       device float [channels][in_row_stride] (needed only for grad_w).
 * grad_w   device float[channels] or NULL to skip; overwritten.
 * The weight gradient is reduced deterministically (no float atomics): two
 * calls with the same inputs give bit-identical results.  With grad_in NULL,
 * on a float plan that offers the 9-trial Tensor-Memory kernel and
 * an `in` that kernel takes (16-byte aligned rows of dd_plan_in_stride), it
 * is computed directly on that kernel's tiles (about twice the forward's
 * time); otherwise from the transpose.  The two ways sum in different orders
 * (both within the float tolerance of the exact result).  Either uses
 * scratch buffers the plan allocates on first use.
 * Errors: DD_ERR_UNSUPPORTED on a uint8 plan, DD_ERR_ARG if both outputs are
 * NULL or grad_w is requested without `in`, DD_ERR_SHAPE, DD_ERR_NOMEM,
 * DD_ERR_CUDA.
 */
dd_status dd_adjoint(dd_plan_t plan, const float* grad_out, int64_t go_row_stride,
                     const float* w, float* grad_in, int64_t gi_row_stride,
                     const float* in, int64_t in_row_stride, float* grad_w, void* stream);

/* ------------------------------------------------------------------- loss */

/*
 * Detection statistic over a dedispersed block (not in the paper; the loss of
 * the differentiable configuration).  For each row i of x ([n_rows][row_stride]
 * float, first n_cols used, n_cols >= 8): boxcar b[t] = sum_{k<8} x[i][t+k] for
 * t in [0, n_cols - 7); mean m_i and population standard deviation s_i of b;
 * S/N z[i][t] = (b[t] - m_i) / s_i.  The maximum of z over (i, t) -- the first
 * one on ties, lowest i then lowest t -- and loss = -max are written to
 * *result (device memory).  Rows with s_i = 0 have no S/N and are skipped;
 * valid = 0 if all are.  If grad (device, [n_rows][grad_stride]) is not NULL
 * it receives d loss / d x: nonzero only in the best row.  Sums are taken in
 * double.  Scratch: n_rows * 32 bytes from the stream-ordered allocator.
 * Errors: DD_ERR_ARG, DD_ERR_SHAPE (n_cols < 8, strides), DD_ERR_NOMEM, DD_ERR_CUDA.
 */
typedef struct {
  double loss;      /* -max S/N */
  double snr;       /* max S/N */
  double mean;      /* boxcar mean of the best row */
  double std;       /* boxcar population standard deviation of the best row */
  int64_t best_t;   /* boxcar start of the maximum */
  int32_t best_row; /* row of the maximum */
  int32_t valid;    /* 0 if every row is constant */
} dd_snr_result;

dd_status dd_boxcar_snr(const float* x, int64_t row_stride, int32_t n_rows, int64_t n_cols,
                        dd_snr_result* result, float* grad, int64_t grad_stride, void* stream);

/*
 * dd_boxcar_snr for callers that must not allocate memory.  The paper has no
 * counterpart: this entry point exists only for how the library is embedded.
 * Some callers cannot call cudaMalloc or any allocator once they are running:
 * a real-time pipeline that reserved all of its device memory at start-up
 * and cannot afford an allocator call (which may synchronise the device or
 * fail) on its hot path, or a host framework that owns every device
 * allocation itself and does not let plug-ins allocate.  This call does the
 * same computation with the same arguments and results as dd_boxcar_snr but
 * allocates nothing: its per-row scratch lives in a fixed array inside the
 * library, DD_NOALLOC_MAX_ROWS rows of 32 bytes (2 MiB), which every GPU that
 * loads the library holds until the process exits.
 *  - n_rows > DD_NOALLOC_MAX_ROWS is rejected with DD_ERR_SHAPE.
 *  - The first call on a device looks up that array's device address (once
 *    per device, with the device current); make that first call before any
 *    stream capture.  The address belongs to the device's context: after
 *    cudaDeviceReset (or anything else that replaces the context) the next
 *    call looks it up again, so that call too should come before any capture.
 *  - Every call on a device shares the one array and it keeps the previous
 *    call's contents; nothing in it needs to start at zero (each call writes
 *    every entry it reads).  Calls that can overlap on the GPU (different
 *    streams, or different host threads on the same device) race on it and
 *    must be serialised by the caller.
 */
#define DD_NOALLOC_MAX_ROWS 65536
dd_status dd_boxcar_snr_noalloc(const float* x, int64_t row_stride, int32_t n_rows, int64_t n_cols,
                                dd_snr_result* result, float* grad, int64_t grad_stride, void* stream);

/* --------------------------------------------------------------- batching */

/*
 * Many independent beams (Section 2: each beam is processed independently;
 * Section 5.1: many beams per device) launched as one CUDA graph.
 * dd_batch_create orders the n plans longest first (C * n_dm * n_out); the
 * plans must outlive the batch and live on the same device.  Mixed uint8 and
 * float32 plans are allowed.
 * dd_batch_run: ins[b] / outs[b] are device pointers for beam b with row
 * strides in_strides[b] / out_strides[b] (host arrays of n entries).  Each
 * beam runs the configuration dd_forward would run for it (its plan's
 * selection, resolved for its input layout) with NULL weights, so results are
 * bit-identical to n separate dd_forward calls.  Beams whose configurations
 * have a persistent form (the staged, packed-uint8 and 9-trial Tensor-Memory
 * kernels) may share one persistent launch per configuration (and blocks per
 * SM; at most 64 beams each): its blocks take the group's tiles, longest beam
 * first, from a work counter until none are left.  Which groups run that way
 * is set by dd_batch_set_persistent; the other beams get one launch each.
 * The launches are dealt to a few internal streams by accumulated work.  The
 * first run on a stream with a given pointer set synchronizes `stream` once,
 * uploads the persistent groups' tensor maps and counters (library-owned
 * device memory) and records the fork from `stream`, the counter resets, the
 * launches and the join into a CUDA graph; later runs with the same pointers
 * replay it with one launch (a run on the legacy NULL stream launches
 * directly).  Work queued on `stream` after the run waits for every beam.
 * Inputs must be 16-byte aligned with 16-byte row pitches (DD_ERR_ALIGN
 * otherwise).  Runs of one batch must not overlap in time (they share the
 * batch's internal streams and device work).  An expired bounded wait in a
 * beam's kernel is reported in that beam's plan status word
 * (dd_plan_device_status; a persistent launch reports it to the beam whose
 * tile timed out and stops).
 */
dd_status dd_batch_create(dd_batch_t* out, const dd_plan_t* plans, int32_t n);
dd_status dd_batch_run(dd_batch_t batch, const void* const* ins, const int64_t* in_strides,
                       void* const* outs, const int64_t* out_strides, void* stream);
/*
 * Auto-tune a batch (Section 2.2 / 4.1: the best configuration depends on the
 * setup): dd_tune (same budget and database rules) runs once per distinct
 * setup of the batch (device, geometry and dtype), longest beams first, and
 * every plan of that setup takes the chosen configuration, so the batch's
 * beams run their tuned kernels.  This changes the plans' selected
 * configurations.  It then times every group of beams that could share a
 * persistent launch against the same beams' own launches (one after another,
 * best of three, on scratch buffers of the largest beam's size, allocated and
 * freed here) and records which form was faster for dd_batch_set_persistent
 * mode 1.  *n_tuned (nullable) receives the number of setups tuned.  The next
 * dd_batch_run records its graph again.
 */
dd_status dd_batch_tune(dd_batch_t batch, double budget_s, const char* db_path, int32_t* n_tuned);
/* Which configuration groups dd_batch_run gives one persistent launch:
 * mode 0: none (one launch per beam); mode 1 (the default): those that
 * dd_batch_tune measured faster than their beams' own launches (none before
 * a tune); mode 2: every group that can have one.  DD_ERR_ARG for another
 * mode.  The next dd_batch_run records its graph again. */
dd_status dd_batch_set_persistent(dd_batch_t batch, int32_t mode);
dd_status dd_batch_destroy(dd_batch_t batch);

/* -------------------------------------------------------------- streaming */

/*
 * Real-time streaming for one beam (Section 4.2: one second of data must be
 * dedispersed in under one second).  The state keeps the last max_delay
 * input samples of every channel on the device, so a stream of chunks of
 * `chunk_len` samples is dedispersed without re-sending the overlap.
 * Chunk k (k = 0, 1, ...) covers input samples [k*N, (k+1)*N), N = chunk_len,
 * and produces output samples [k*N - max_delay, (k+1)*N - max_delay):
 * *out_t0 receives k*N - max_delay.  The tail starts zero-filled, so outputs
 * at negative times include those zeros; every output at time >= 0 equals
 * dd_forward on the concatenated input.
 * chunk  device [channels][chunk_len] (element type of the plan), contiguous.
 * out    device [n_dm][chunk_len] of the plan's output type, contiguous.
 * The plan's n_out is not used by streaming; the output length is chunk_len.
 * dd_stream_save / dd_stream_restore copy the state (tail + sample counter)
 * to / from a host buffer of dd_stream_state_bytes bytes, for checkpointing.
 * dd_stream_reset zeroes the tail on `stream` (asynchronously, ordered after
 * the pushes queued on that stream) and restarts the chunk count at 0; pushes
 * on other streams must be ordered against it by the caller.
 */
dd_status dd_stream_create(dd_stream_t* out, dd_plan_t plan, int64_t chunk_len);
dd_status dd_stream_push(dd_stream_t st, const void* chunk, void* out, int64_t* out_t0, void* stream);
dd_status dd_stream_reset(dd_stream_t st, void* stream);
dd_status dd_stream_state_bytes(dd_stream_t st, int64_t* bytes);
/* Device bytes the stream holds: its own plan's tables (the geometry with
 * n_out = chunk_len) and its two state buffers.  dd_stream_footprint reports
 * the same number for a geometry before any stream exists (host-only;
 * arguments and errors as dd_plan and dd_stream_create). */
dd_status dd_stream_device_bytes(dd_stream_t st, int64_t* bytes);
dd_status dd_stream_footprint(int32_t channels, double f_low_mhz, double chan_bw_mhz, double t_samp_s,
                              double dm_first, double dm_step, int32_t n_dm, int64_t chunk_len, dd_dtype dtype,
                              int64_t* device_bytes);
dd_status dd_stream_save(dd_stream_t st, void* host_buf, void* stream);
dd_status dd_stream_restore(dd_stream_t st, const void* host_buf, void* stream);
dd_status dd_stream_destroy(dd_stream_t st);

/* --------------------------------------------------------------- tuning */

/*
 * Auto-tuning (Section 2.2, last paragraph; Section 4.1): times every valid
 * tile configuration of the plan on synthetic data with CUDA events (median of
 * repeated launches) and selects the fastest, within `budget_s` seconds of
 * wall time (0 = no limit).  If db_path is not NULL the choice is recorded in
 * that JSON-lines file (one line per call: device name, plan geometry, dtype,
 * config name, time) and an existing entry for the same key is reused without
 * timing.  Allocates and frees its own device buffers; synchronises the
 * device.  *best_ms (nullable) receives the selected config's median time.
 * A plan created while the environment variable DD_TUNE_DB names such a file
 * starts with the choice recorded there for its device and geometry, if any.
 */
dd_status dd_tune(dd_plan_t plan, double budget_s, const char* db_path, double* best_ms);

/* ----------------------------------------------------------------- errors */

/* Static name of a status code. */
const char* dd_status_string(dd_status s);
/* Detail of the last failing call on this thread ("" if none).  Valid until
 * the next failing call on the same thread. */
const char* dd_last_error(void);
/* Library version string. */
const char* dd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBDD_DD_H */
