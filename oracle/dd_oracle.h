/*
 * dd_oracle.h -- plain CPU reference for brute-force incoherent dedispersion.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the parity authority for the
 * CUDA path: it is slow on purpose, written as the paper's definitions
 * (Eq. 1 delay law, Eq. 3 direct transform, Algorithm 1 triple loop) with
 * FP64 arithmetic and no blocking, fusion or reordering.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no source, header, table or constant with the CUDA library.
 *
 * Conventions (readings of the paper, each argued in the design notes):
 *   - C_DM = 4148.808 MHz^2 s pc^-1 cm^3 (Eq. 1 prints a garbled constant).
 *   - Per-channel delay coefficient k_c = C_DM * (1/f_c^2 - 1/f_ref^2) [s per
 *     unit DM] (Eq. 1 with f_low = f_c, f_high = f_ref; Eq. 7 form).
 *   - Shift s(c,d) = floor(DM_d * k_c / (bin * t_samp) + 0.5)  (round half up).
 *   - DM grid per range: DM_d = lo + d*step, n_dm = llround((hi-lo)/step)
 *     (fixed step per range, half-open; Table 2 trial counts).
 *   - Decimation by `bin`: X_b[c][t'] = sum_{j<bin} X[c][bin*t'+j]; the tail
 *     of n_samp mod bin samples is dropped.
 *   - Valid-only outputs: N_out = floor(n_samp/bin) - S_max, S_max = max s.
 *   - Raw sums, no normalisation.
 *
 * All functions return 0 on success and a negative code on bad arguments.
 */
#ifndef DD_ORACLE_H
#define DD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_DTYPE_U8 1
#define ORACLE_DTYPE_U16 2
#define ORACLE_DTYPE_F32 3
#define ORACLE_DTYPE_U4 4  /* two samples per byte, the earlier one in the low nibble */

typedef struct {
  double dm_lo;   /* first trial DM, pc cm^-3 */
  double dm_hi;   /* end of the half-open DM range */
  double dm_step; /* fixed DM step of the range */
  int32_t bin;    /* time decimation factor (>= 1) */
} oracle_range;

/* Dispersion constant used throughout (Eq. 1). */
double oracle_c_dm(void);

/* Number of trial DMs of a range: llround((hi - lo) / step). */
int64_t oracle_range_ndm(oracle_range r);

/* Trial DM number d of a range: lo + d*step (a product, never a running sum). */
double oracle_range_dm(oracle_range r, int64_t d);

/* Eq. 1 delay per unit DM of a channel at f_mhz relative to f_ref_mhz [s]. */
double oracle_delay_coeff(double f_mhz, double f_ref_mhz);

/* Integer shift of one (channel, DM) in decimated samples. */
int64_t oracle_shift(double dm, double k_c, int32_t bin, double t_samp_s);

/* Full shift table of one range: out[d * n_chan + c] = s(c, d). */
int oracle_shift_table(const double* freqs_mhz, int32_t n_chan, double f_ref_mhz,
                       double t_samp_s, oracle_range r, int64_t* out);

/* Largest shift of a range and its output length for n_samp raw samples.
 * n_out <= 0 means the range is too long for the input. */
int oracle_range_extent(const double* freqs_mhz, int32_t n_chan, double f_ref_mhz,
                        double t_samp_s, oracle_range r, int64_t n_samp,
                        int64_t* s_max, int64_t* n_out);

/*
 * Direct transform (Eq. 3, Algorithm 1) of one range on selected DM rows and a
 * time window [t_begin, t_end) of output samples:
 *   out[i][t - t_begin] = sum_c X_b[c][t + s(c, rows[i])]
 * x is channel-major [n_chan][row_stride] of the given dtype (row_stride and
 * n_samp count samples; 4-bit rows are row_stride / 2 bytes).  Integer inputs
 * are summed in int64, float inputs in FP64; out is FP64 in both cases (every
 * integer sum here is far below 2^53).  If take_abs is non-zero, |X| is summed
 * instead (used for the float tolerance bound).  OpenMP over rows.
 */
int oracle_forward_rows(int dtype, const void* x, int32_t n_chan, int64_t n_samp,
                        int64_t row_stride, const double* freqs_mhz, double f_ref_mhz,
                        double t_samp_s, oracle_range r, const int64_t* rows,
                        int64_t n_rows, int64_t t_begin, int64_t t_end, int take_abs,
                        double* out);

/* Whole plan: out is the concatenation over ranges of [n_dm_r][N_out_r]. */
int oracle_forward(int dtype, const void* x, int32_t n_chan, int64_t n_samp,
                   int64_t row_stride, const double* freqs_mhz, double f_ref_mhz,
                   double t_samp_s, const oracle_range* ranges, int32_t n_ranges,
                   int take_abs, double* out);

/*
 * Transpose of the whole-plan forward map (re-dispersion):
 *   xbar[c][t] = sum_r sum_d ybar_r[d][floor(t/b_r) - s_r(c,d)]
 * over the terms with 0 <= floor(t/b_r) - s_r(c,d) < N_out_r and
 * floor(t/b_r) < floor(n_samp/b_r).  ybar is the concatenated output layout
 * (FP64), xbar is [n_chan][n_samp] FP64 and is overwritten.  Written as the
 * scatter of each output back along its dispersion track.
 */
int oracle_adjoint(const double* ybar, int32_t n_chan, int64_t n_samp,
                   const double* freqs_mhz, double f_ref_mhz, double t_samp_s,
                   const oracle_range* ranges, int32_t n_ranges, double* xbar);

/* The same transpose for the channels listed in chans[n_sel] only:
 * xbar[i][t] is channel chans[i] of the full result (the plan's extents still
 * come from all n_chan channels). */
int oracle_adjoint_channels(const double* ybar, int32_t n_chan, int64_t n_samp,
                            const double* freqs_mhz, double f_ref_mhz, double t_samp_s,
                            const oracle_range* ranges, int32_t n_ranges, const int32_t* chans,
                            int32_t n_sel, double* xbar);

/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
int oracle_threads(void);

#ifdef __cplusplus
}
#endif

#endif /* DD_ORACLE_H */
