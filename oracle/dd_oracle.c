/*
 * Oracle for brute-force incoherent dedispersion (Sclocco et al., "Real-Time
 * Dedispersion for Fast Radio Transient Surveys, using Auto Tuning on
 * Many-Core Accelerators").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the library computes.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant with the CUDA library: the
 * library has its own delay-table code, and the two are compared in tests.
 *
 * Every loop below follows the paper's definition in the paper's order, with
 * no blocking, fusion or reordering:
 *   - delay table: Eq. 1 (Section 2), turned into whole samples by rounding
 *     half up (the paper is silent on rounding; see the readings list in the
 *     design notes);
 *   - forward: Algorithm 1 (Section 2.1), three nested loops dm -> sample ->
 *     channel, with an optional per-channel weight;
 *   - adjoint and weight gradient: the transpose of Algorithm 1 and its
 *     derivative with respect to the weights (not in the paper);
 *   - boxcar / S/N loss: an 8-sample boxcar, per-DM standardisation and a
 *     hard maximum (not in the paper).
 * Floating point is accumulated in double (fp64), 8-bit input in int64.
 *
 * Parity pins: every function here is pinned by tests that do not call it
 * back (see tests/test_oracle_pins.py).  No function is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

/* Return codes (oracle-local; unrelated to the library's status codes). */
#define ORC_OK 0
#define ORC_EARG 1
#define ORC_ERANGE 2

/*
 * Eq. 1: the delay, in seconds, of frequency f_i relative to the highest
 * frequency f_h of the band is 4150 * DM * (1/f_i^2 - 1/f_h^2), frequencies in
 * MHz.  Channel c has centre frequency f_low + c * chan_bw (channel 0 lowest),
 * f_h is the top channel's frequency, DM trial i is dm_first + i * dm_step.
 * The delay in samples is the delay in seconds divided by the sampling time,
 * rounded half up.  d is [n_dm][C], row-major.
 */
int orc_delay_table(int32_t C, double f_low, double chan_bw, double t_samp,
                    double dm_first, double dm_step, int32_t n_dm, int32_t* d) {
  if (C <= 0 || n_dm <= 0 || !(f_low > 0.0) || !(chan_bw > 0.0) || !(t_samp > 0.0) ||
      !(dm_first >= 0.0) || !(dm_step >= 0.0) || d == NULL)
    return ORC_EARG;
  double f_h = f_low + (double)(C - 1) * chan_bw;
  for (int32_t i = 0; i < n_dm; ++i) {
    double dm = dm_first + (double)i * dm_step;
    for (int32_t c = 0; c < C; ++c) {
      double f_i = f_low + (double)c * chan_bw;
      double k_seconds = (4150.0 * dm) * (1.0 / (f_i * f_i) - 1.0 / (f_h * f_h));
      double samples = k_seconds / t_samp;
      double rounded = floor(samples + 0.5);
      if (rounded > 2147483647.0) return ORC_ERANGE;
      d[(size_t)i * C + c] = (int32_t)rounded;
    }
  }
  return ORC_OK;
}

/* Largest delay in the table: the lowest channel at the highest DM trial. */
int32_t orc_max_delay(const int32_t* d, int32_t C, int32_t n_dm) {
  int32_t m = 0;
  for (int64_t k = 0; k < (int64_t)C * n_dm; ++k)
    if (d[k] > m) m = d[k];
  return m;
}

/*
 * Algorithm 1 on 32-bit float input: out[dm][sample] =
 * sum over chan of w[chan] * input[chan][sample + delay(chan, dm)], summed in
 * double.  w may be NULL (all weights 1).  in is [C][n_in], out is
 * [n_dm][n_out]; n_in must be at least n_out + max delay.
 */
int orc_forward_f32(int32_t C, int32_t n_dm, int64_t n_out, int64_t n_in,
                    const int32_t* d, const float* in, const float* w, double* out) {
  if (n_in < n_out + orc_max_delay(d, C, n_dm)) return ORC_EARG;
  for (int32_t dm = 0; dm < n_dm; ++dm) {
    for (int64_t sample = 0; sample < n_out; ++sample) {
      double dsample = 0.0;
      for (int32_t chan = 0; chan < C; ++chan) {
        double weight = w ? (double)w[chan] : 1.0;
        int64_t shift = d[(size_t)dm * C + chan];
        dsample += weight * (double)in[(size_t)chan * n_in + sample + shift];
      }
      out[(size_t)dm * n_out + sample] = dsample;
    }
  }
  return ORC_OK;
}

/*
 * Algorithm 1 on unsigned 8-bit input with unit weights, summed in int64 and
 * stored as int32 (the sum of C values of at most 255 must fit).
 */
int orc_forward_u8(int32_t C, int32_t n_dm, int64_t n_out, int64_t n_in,
                   const int32_t* d, const uint8_t* in, int32_t* out) {
  if (n_in < n_out + orc_max_delay(d, C, n_dm)) return ORC_EARG;
  for (int32_t dm = 0; dm < n_dm; ++dm) {
    for (int64_t sample = 0; sample < n_out; ++sample) {
      int64_t dsample = 0;
      for (int32_t chan = 0; chan < C; ++chan) {
        int64_t shift = d[(size_t)dm * C + chan];
        dsample += (int64_t)in[(size_t)chan * n_in + sample + shift];
      }
      if (dsample > 2147483647LL) return ORC_ERANGE;
      out[(size_t)dm * n_out + sample] = (int32_t)dsample;
    }
  }
  return ORC_OK;
}

/*
 * Transpose of Algorithm 1 (not in the paper).  Algorithm 1 reads
 * input[chan][sample + delay] once per (dm, sample, chan) with weight w[chan];
 * its adjoint sends grad_out[dm][sample] back to that same input position:
 *   grad_in[chan][u] = sum over dm of w[chan] * grad_out[dm][u - delay(chan, dm)]
 * over the dm for which 0 <= u - delay < n_out; every other position is 0.
 * Written as the scatter it is, in Algorithm 1's loop order.
 */
int orc_adjoint_f32(int32_t C, int32_t n_dm, int64_t n_out, int64_t n_in,
                    const int32_t* d, const float* grad_out, const float* w, double* grad_in) {
  if (n_in < n_out + orc_max_delay(d, C, n_dm)) return ORC_EARG;
  for (int64_t k = 0; k < (int64_t)C * n_in; ++k) grad_in[k] = 0.0;
  for (int32_t dm = 0; dm < n_dm; ++dm) {
    for (int64_t sample = 0; sample < n_out; ++sample) {
      double g = (double)grad_out[(size_t)dm * n_out + sample];
      for (int32_t chan = 0; chan < C; ++chan) {
        double weight = w ? (double)w[chan] : 1.0;
        int64_t shift = d[(size_t)dm * C + chan];
        grad_in[(size_t)chan * n_in + sample + shift] += weight * g;
      }
    }
  }
  return ORC_OK;
}

/*
 * Derivative of the weighted Algorithm 1 with respect to w[chan] (not in the
 * paper): grad_w[chan] = sum over dm, sample of
 * grad_out[dm][sample] * input[chan][sample + delay(chan, dm)].
 */
int orc_wgrad_f32(int32_t C, int32_t n_dm, int64_t n_out, int64_t n_in,
                  const int32_t* d, const float* grad_out, const float* in, double* grad_w) {
  if (n_in < n_out + orc_max_delay(d, C, n_dm)) return ORC_EARG;
  for (int32_t chan = 0; chan < C; ++chan) grad_w[chan] = 0.0;
  for (int32_t dm = 0; dm < n_dm; ++dm) {
    for (int64_t sample = 0; sample < n_out; ++sample) {
      double g = (double)grad_out[(size_t)dm * n_out + sample];
      for (int32_t chan = 0; chan < C; ++chan) {
        int64_t shift = d[(size_t)dm * C + chan];
        grad_w[chan] += g * (double)in[(size_t)chan * n_in + sample + shift];
      }
    }
  }
  return ORC_OK;
}

/*
 * Detection loss on a dedispersed block (not in the paper).  For each DM
 * trial i: boxcar b[t] = sum_{k<8} out[i][t+k] for t in [0, n_out-7);
 * mean m_i and population standard deviation s_i of b over t;
 * snr[i][t] = (b[t] - m_i) / s_i.  loss = -max over (i, t) of snr, the first
 * (lowest i, then lowest t) maximum on ties.  If grad_out is not NULL it
 * receives d loss / d out[i][t] ([n_dm][n_out], zero outside row i*), using
 *   d snr[t*] / d b[t] = ((t == t*) - 1/n) / s - snr[t*] * snr[t] / (n * s).
 * best_i / best_t (nullable) receive the arg-max.  Rows with s == 0 have no
 * defined S/N and are skipped; if every row is constant, ORC_ERANGE.
 */
int orc_boxcar_snr_loss(int32_t n_dm, int64_t n_out, const double* out, double* loss,
                        double* grad_out, int32_t* best_i, int64_t* best_t) {
  const int64_t W = 8;
  if (n_out < W || n_dm <= 0) return ORC_EARG;
  int64_t nb = n_out - W + 1;
  double best = -INFINITY;
  int32_t bi = -1;
  int64_t bt = -1;
  double b_mean = 0.0, b_std = 0.0;
  for (int32_t i = 0; i < n_dm; ++i) {
    const double* row = out + (size_t)i * n_out;
    double sum = 0.0;
    for (int64_t t = 0; t < nb; ++t) {
      double b = 0.0;
      for (int64_t k = 0; k < W; ++k) b += row[t + k];
      sum += b;
    }
    double mean = sum / (double)nb;
    double var = 0.0;
    for (int64_t t = 0; t < nb; ++t) {
      double b = 0.0;
      for (int64_t k = 0; k < W; ++k) b += row[t + k];
      var += (b - mean) * (b - mean);
    }
    var /= (double)nb;
    double sd = sqrt(var);
    if (!(sd > 0.0)) continue;
    for (int64_t t = 0; t < nb; ++t) {
      double b = 0.0;
      for (int64_t k = 0; k < W; ++k) b += row[t + k];
      double snr = (b - mean) / sd;
      if (snr > best) {
        best = snr;
        bi = i;
        bt = t;
        b_mean = mean;
        b_std = sd;
      }
    }
  }
  if (bi < 0) return ORC_ERANGE;
  *loss = -best;
  if (best_i) *best_i = bi;
  if (best_t) *best_t = bt;
  if (grad_out) {
    for (int64_t k = 0; k < (int64_t)n_dm * n_out; ++k) grad_out[k] = 0.0;
    const double* row = out + (size_t)bi * n_out;
    double* grow = grad_out + (size_t)bi * n_out;
    double zstar = best;
    for (int64_t t = 0; t < nb; ++t) {
      double b = 0.0;
      for (int64_t k = 0; k < W; ++k) b += row[t + k];
      double z = (b - b_mean) / b_std;
      double dz_db = ((t == bt ? 1.0 : 0.0) - 1.0 / (double)nb) / b_std -
                     zstar * z / ((double)nb * b_std);
      /* loss = -snr[t*]; b[t] depends on out[t..t+7] with unit weight. */
      for (int64_t k = 0; k < W; ++k) grow[t + k] += -dz_db;
    }
  }
  return ORC_OK;
}
