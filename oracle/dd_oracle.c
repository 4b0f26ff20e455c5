/*
 * dd_oracle.c -- plain CPU reference for brute-force incoherent dedispersion.
 *
 * TEST INFRASTRUCTURE ONLY (see dd_oracle.h).  Every function is the paper's
 * definition written out with plain loops in FP64 / int64:
 *   - oracle_delay_coeff: Eq. 1 (cold-plasma delay law), per-channel form of
 *     Eq. 7 (Sec. 4.1, Delta t_pc).
 *   - oracle_shift: the integer shift of Eq. 3, rounded half up.
 *   - oracle_forward_rows: Eq. 3 / Algorithm 1 (Sec. 2), the triple loop over
 *     time, DM and channel, with the per-range time binning of Sec. 5.3.
 *   - oracle_adjoint: the transpose of that linear map.
 * Build with -ffp-contract=off and without -ffast-math so that the FP64
 * expressions below are evaluated exactly as written on every host.
 */
#include "dd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Eq. 1 dispersion constant in MHz^2 s pc^-1 cm^3 (the paper prints it with a
 * garbled power of ten; 4148.808 is the value the method is specified with). */
static const double kCdm = 4148.808;

double oracle_c_dm(void) { return kCdm; }

int64_t oracle_range_ndm(oracle_range r) {
  if (!(r.dm_step > 0.0) || !(r.dm_hi > r.dm_lo)) return 0;
  return (int64_t)llround((r.dm_hi - r.dm_lo) / r.dm_step);
}

double oracle_range_dm(oracle_range r, int64_t d) {
  return r.dm_lo + (double)d * r.dm_step;
}

double oracle_delay_coeff(double f_mhz, double f_ref_mhz) {
  /* Eq. 1 with f_low = f, f_high = f_ref: C_DM * (1/f^2 - 1/f_ref^2). */
  double inv_f2 = 1.0 / (f_mhz * f_mhz);
  double inv_ref2 = 1.0 / (f_ref_mhz * f_ref_mhz);
  return kCdm * (inv_f2 - inv_ref2);
}

int64_t oracle_shift(double dm, double k_c, int32_t bin, double t_samp_s) {
  /* Delay in units of the (decimated) sample time, rounded half up. */
  double delay = dm * k_c;
  double tick = (double)bin * t_samp_s;
  double x = delay / tick;
  return (int64_t)floor(x + 0.5);
}

static int check_plan(const double* freqs_mhz, int32_t n_chan, double f_ref_mhz,
                      double t_samp_s, oracle_range r) {
  if (!freqs_mhz || n_chan <= 0) return -1;
  if (!(t_samp_s > 0.0) || !(f_ref_mhz > 0.0)) return -1;
  if (r.bin < 1 || oracle_range_ndm(r) <= 0 || r.dm_lo < 0.0) return -1;
  for (int32_t c = 0; c < n_chan; ++c) {
    if (!(freqs_mhz[c] > 0.0) || freqs_mhz[c] > f_ref_mhz) return -1;
  }
  return 0;
}

int oracle_shift_table(const double* freqs_mhz, int32_t n_chan, double f_ref_mhz,
                       double t_samp_s, oracle_range r, int64_t* out) {
  if (check_plan(freqs_mhz, n_chan, f_ref_mhz, t_samp_s, r) != 0 || !out) return -1;
  int64_t n_dm = oracle_range_ndm(r);
  for (int64_t d = 0; d < n_dm; ++d) {
    double dm = oracle_range_dm(r, d);
    for (int32_t c = 0; c < n_chan; ++c) {
      double k_c = oracle_delay_coeff(freqs_mhz[c], f_ref_mhz);
      out[d * n_chan + c] = oracle_shift(dm, k_c, r.bin, t_samp_s);
    }
  }
  return 0;
}

int oracle_range_extent(const double* freqs_mhz, int32_t n_chan, double f_ref_mhz,
                        double t_samp_s, oracle_range r, int64_t n_samp,
                        int64_t* s_max, int64_t* n_out) {
  if (check_plan(freqs_mhz, n_chan, f_ref_mhz, t_samp_s, r) != 0) return -1;
  if (n_samp < 0 || !s_max || !n_out) return -1;
  int64_t n_dm = oracle_range_ndm(r);
  int64_t smax = 0;
  for (int64_t d = 0; d < n_dm; ++d) {
    double dm = oracle_range_dm(r, d);
    for (int32_t c = 0; c < n_chan; ++c) {
      int64_t s = oracle_shift(dm, oracle_delay_coeff(freqs_mhz[c], f_ref_mhz),
                               r.bin, t_samp_s);
      if (s > smax) smax = s;
    }
  }
  *s_max = smax;
  *n_out = n_samp / r.bin - smax;
  return 0;
}

/* One raw sample as int64.  idx counts samples; 4-bit samples are packed two
 * per byte, sample 2k in the low nibble of byte k and 2k+1 in the high one. */
static inline int64_t load_int(int dtype, const void* x, int64_t idx) {
  if (dtype == ORACLE_DTYPE_U8) return (int64_t)((const uint8_t*)x)[idx];
  if (dtype == ORACLE_DTYPE_U4) {
    const uint8_t byte = ((const uint8_t*)x)[idx / 2];
    return (int64_t)((idx % 2 == 0) ? (byte & 0x0f) : (byte >> 4));
  }
  return (int64_t)((const uint16_t*)x)[idx];
}

int oracle_forward_rows(int dtype, const void* x, int32_t n_chan, int64_t n_samp,
                        int64_t row_stride, const double* freqs_mhz, double f_ref_mhz,
                        double t_samp_s, oracle_range r, const int64_t* rows,
                        int64_t n_rows, int64_t t_begin, int64_t t_end, int take_abs,
                        double* out) {
  if (dtype != ORACLE_DTYPE_U8 && dtype != ORACLE_DTYPE_U16 && dtype != ORACLE_DTYPE_F32 &&
      dtype != ORACLE_DTYPE_U4)
    return -1;
  if (!x || !rows || !out || n_rows < 0 || row_stride < n_samp) return -1;
  if (dtype == ORACLE_DTYPE_U4 && row_stride % 2 != 0) return -1;
  int64_t s_max = 0, n_out = 0;
  if (oracle_range_extent(freqs_mhz, n_chan, f_ref_mhz, t_samp_s, r, n_samp, &s_max,
                          &n_out) != 0)
    return -1;
  if (n_out <= 0 || t_begin < 0 || t_end > n_out || t_begin > t_end) return -2;
  int64_t n_dm = oracle_range_ndm(r);
  for (int64_t i = 0; i < n_rows; ++i)
    if (rows[i] < 0 || rows[i] >= n_dm) return -1;

  const int64_t width = t_end - t_begin;
  const int32_t b = r.bin;
  int failed = 0;

#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n_rows; ++i) {
    double dm = oracle_range_dm(r, rows[i]);
    double* orow = out + i * width;
    if (dtype == ORACLE_DTYPE_F32) {
      double* acc = (double*)calloc((size_t)(width > 0 ? width : 1), sizeof(double));
      if (!acc) { failed = 1; continue; }
      for (int32_t c = 0; c < n_chan; ++c) {
        int64_t s = oracle_shift(dm, oracle_delay_coeff(freqs_mhz[c], f_ref_mhz), b,
                                 t_samp_s);
        const float* xc = (const float*)x + (int64_t)c * row_stride;
        for (int64_t t = t_begin; t < t_end; ++t) {
          /* X_b[c][t + s]: the sum of the bin raw samples it covers. */
          for (int32_t j = 0; j < b; ++j) {
            double v = (double)xc[(t + s) * b + j];
            acc[t - t_begin] += take_abs ? fabs(v) : v;
          }
        }
      }
      for (int64_t t = 0; t < width; ++t) orow[t] = acc[t];
      free(acc);
    } else {
      int64_t* acc = (int64_t*)calloc((size_t)(width > 0 ? width : 1), sizeof(int64_t));
      if (!acc) { failed = 1; continue; }
      for (int32_t c = 0; c < n_chan; ++c) {
        int64_t s = oracle_shift(dm, oracle_delay_coeff(freqs_mhz[c], f_ref_mhz), b,
                                 t_samp_s);
        int64_t base = (int64_t)c * row_stride;
        for (int64_t t = t_begin; t < t_end; ++t) {
          for (int32_t j = 0; j < b; ++j) acc[t - t_begin] += load_int(dtype, x, base + (t + s) * b + j);
        }
      }
      for (int64_t t = 0; t < width; ++t) orow[t] = (double)acc[t];
      free(acc);
    }
  }
  return failed ? -3 : 0;
}

int oracle_forward(int dtype, const void* x, int32_t n_chan, int64_t n_samp,
                   int64_t row_stride, const double* freqs_mhz, double f_ref_mhz,
                   double t_samp_s, const oracle_range* ranges, int32_t n_ranges,
                   int take_abs, double* out) {
  if (!ranges || n_ranges <= 0 || !out) return -1;
  int64_t offset = 0;
  for (int32_t k = 0; k < n_ranges; ++k) {
    int64_t s_max = 0, n_out = 0;
    if (oracle_range_extent(freqs_mhz, n_chan, f_ref_mhz, t_samp_s, ranges[k], n_samp,
                            &s_max, &n_out) != 0)
      return -1;
    if (n_out <= 0) return -2;
    int64_t n_dm = oracle_range_ndm(ranges[k]);
    int64_t* rows = (int64_t*)malloc((size_t)n_dm * sizeof(int64_t));
    if (!rows) return -3;
    for (int64_t d = 0; d < n_dm; ++d) rows[d] = d;
    int rc = oracle_forward_rows(dtype, x, n_chan, n_samp, row_stride, freqs_mhz,
                                 f_ref_mhz, t_samp_s, ranges[k], rows, n_dm, 0, n_out,
                                 take_abs, out + offset);
    free(rows);
    if (rc != 0) return rc;
    offset += n_dm * n_out;
  }
  return 0;
}

/* Transpose for a list of channels (all channels when chans is NULL). */
static int adjoint_impl(const double* ybar, int32_t n_chan, int64_t n_samp,
                        const double* freqs_mhz, double f_ref_mhz, double t_samp_s,
                        const oracle_range* ranges, int32_t n_ranges, const int32_t* chans,
                        int32_t n_sel, double* xbar) {
  if (!ybar || !xbar || !ranges || n_ranges <= 0 || n_samp <= 0 || n_sel < 0) return -1;
  int64_t* n_outs = (int64_t*)malloc((size_t)n_ranges * sizeof(int64_t));
  int64_t* offsets = (int64_t*)malloc((size_t)n_ranges * sizeof(int64_t));
  if (!n_outs || !offsets) { free(n_outs); free(offsets); return -3; }
  int64_t offset = 0;
  for (int32_t k = 0; k < n_ranges; ++k) {
    int64_t s_max = 0, n_out = 0;
    if (oracle_range_extent(freqs_mhz, n_chan, f_ref_mhz, t_samp_s, ranges[k], n_samp,
                            &s_max, &n_out) != 0 || n_out <= 0) {
      free(n_outs); free(offsets);
      return n_out <= 0 ? -2 : -1;
    }
    n_outs[k] = n_out;
    offsets[k] = offset;
    offset += oracle_range_ndm(ranges[k]) * n_out;
  }
  for (int32_t i = 0; i < n_sel; ++i) {
    if (chans && (chans[i] < 0 || chans[i] >= n_chan)) { free(n_outs); free(offsets); return -1; }
  }
  memset(xbar, 0, (size_t)n_sel * (size_t)n_samp * sizeof(double));

  /* Each output Y_r[d][t] read X[c][b*(t+s)+j] for j < b: send its cotangent
   * back to exactly those inputs.  Channels are independent. */
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t i = 0; i < n_sel; ++i) {
    const int32_t c = chans ? chans[i] : i;
    double* xc = xbar + (int64_t)i * n_samp;
    for (int32_t k = 0; k < n_ranges; ++k) {
      oracle_range r = ranges[k];
      int64_t n_dm = oracle_range_ndm(r);
      double k_c = oracle_delay_coeff(freqs_mhz[c], f_ref_mhz);
      for (int64_t d = 0; d < n_dm; ++d) {
        int64_t s = oracle_shift(oracle_range_dm(r, d), k_c, r.bin, t_samp_s);
        const double* yrow = ybar + offsets[k] + d * n_outs[k];
        for (int64_t t = 0; t < n_outs[k]; ++t) {
          for (int32_t j = 0; j < r.bin; ++j) xc[(t + s) * r.bin + j] += yrow[t];
        }
      }
    }
  }
  free(n_outs);
  free(offsets);
  return 0;
}

int oracle_adjoint(const double* ybar, int32_t n_chan, int64_t n_samp,
                   const double* freqs_mhz, double f_ref_mhz, double t_samp_s,
                   const oracle_range* ranges, int32_t n_ranges, double* xbar) {
  return adjoint_impl(ybar, n_chan, n_samp, freqs_mhz, f_ref_mhz, t_samp_s, ranges, n_ranges,
                      NULL, n_chan, xbar);
}

int oracle_adjoint_channels(const double* ybar, int32_t n_chan, int64_t n_samp,
                            const double* freqs_mhz, double f_ref_mhz, double t_samp_s,
                            const oracle_range* ranges, int32_t n_ranges, const int32_t* chans,
                            int32_t n_sel, double* xbar) {
  if (!chans) return -1;
  return adjoint_impl(ybar, n_chan, n_samp, freqs_mhz, f_ref_mhz, t_samp_s, ranges, n_ranges,
                      chans, n_sel, xbar);
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
