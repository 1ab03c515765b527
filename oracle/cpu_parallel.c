/*
 * Multi-threaded CPU baseline of Algorithm 1 (the paper's CPU comparison,
 * Section 5): the oracle's sum, spread over the host's cores with OpenMP.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the rest of this directory:
 * only the tests and the benchmark's CPU-baseline leg load it.
 *
 * Each output element is the same fp64 sum as in dd_oracle.c, over channels
 * in ascending order (so the two agree bit for bit; the tests check it).
 * What differs is the loop nest: DM trials are shared among threads in
 * chunks of `dm_chunk`, and within a trial time runs in blocks of `t_block`
 * samples with the channel loop outside the sample loop, so that a block of
 * partial sums stays in cache and the inner loop is a contiguous vectorisable
 * sweep.  `threads` and the two block sizes are the knobs a tuner varies.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CPB_OK 0
#define CPB_EARG 1
#define CPB_ENOMEM 2

/* Number of threads OpenMP would use (1 without OpenMP). */
int cpb_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int cpb_forward_f32(int32_t C, int32_t n_dm, int64_t n_out, int64_t n_in, const int32_t* d, const float* in,
                    const float* w, double* out, int32_t threads, int32_t dm_chunk, int32_t t_block) {
  if (C <= 0 || n_dm <= 0 || n_out <= 0 || dm_chunk <= 0 || t_block <= 0) return CPB_EARG;
  for (int64_t k = 0; k < (int64_t)n_dm * C; ++k)
    if (d[k] < 0 || d[k] + n_out > n_in) return CPB_EARG;
  int failed = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
#endif
  {
    double* acc = (double*)malloc(sizeof(double) * (size_t)t_block);
    if (!acc) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      failed = 1;
    }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int32_t dm0 = 0; dm0 < n_dm; dm0 += dm_chunk) {
      if (!acc) continue;
      const int32_t dm1 = dm0 + dm_chunk < n_dm ? dm0 + dm_chunk : n_dm;
      for (int32_t dm = dm0; dm < dm1; ++dm) {
        const int32_t* dd = d + (size_t)dm * C;
        for (int64_t t0 = 0; t0 < n_out; t0 += t_block) {
          const int64_t nt = t0 + t_block < n_out ? t_block : n_out - t0;
          for (int64_t t = 0; t < nt; ++t) acc[t] = 0.0;
          for (int32_t chan = 0; chan < C; ++chan) {
            const double weight = w ? (double)w[chan] : 1.0;
            const float* src = in + (size_t)chan * n_in + t0 + dd[chan];
            for (int64_t t = 0; t < nt; ++t) acc[t] += weight * (double)src[t];
          }
          double* dst = out + (size_t)dm * n_out + t0;
          for (int64_t t = 0; t < nt; ++t) dst[t] = acc[t];
        }
      }
    }
    free(acc);
  }
  return failed ? CPB_ENOMEM : CPB_OK;
}
