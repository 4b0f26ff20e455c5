/*
 * synth.c -- seeded synthetic filterbank generator shared by the tests, the
 * oracle checks and the benchmark.  It holds none of the dedispersion
 * arithmetic: pulse tracks arrive as per-channel start samples computed by the
 * caller.
 *
 * Noise is counter based, so any element can be produced independently:
 *   - splitmix64 (Steele, Lea and Flood, OOPSLA 2014): output n of a stream
 *     with seed S is mix(S + n * 0x9E3779B97F4A7C15), n = 1, 2, ...
 *   - Box-Muller (Box and Muller, 1958): uniforms u1 in (0, 1] and u2 in
 *     [0, 1) from outputs 2p+1 and 2p+2 give the normal pair
 *     (r cos(2 pi u2), r sin(2 pi u2)), r = sqrt(-2 ln u1), for the global
 *     elements 2p and 2p+1 (element index i = channel * n_samp + sample).
 * Integer samples are clamp(floor(mean + sd*z + pulses + 0.5), lo, hi); float
 * samples are (float)(mean + sd*z + pulses).  Pulses are boxcars of width w
 * and amplitude a starting at start[c] in channel c, added before rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t synth_splitmix64(uint64_t seed, uint64_t n) { return mix64(seed + n * kGamma); }

/* Normal variate of global element i of stream `seed`. */
static inline double normal_at(uint64_t seed, uint64_t i, uint64_t* cached_p,
                               double* cached_r, double* cached_th) {
  uint64_t p = i >> 1;
  if (p != *cached_p) {
    uint64_t h1 = mix64(seed + (2 * p + 1) * kGamma);
    uint64_t h2 = mix64(seed + (2 * p + 2) * kGamma);
    double u1 = (double)((h1 >> 11) + 1) * (1.0 / 9007199254740992.0);
    double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
    *cached_r = sqrt(-2.0 * log(u1));
    *cached_th = 6.283185307179586 * u2;
    *cached_p = p;
  }
  return (i & 1) ? *cached_r * sin(*cached_th) : *cached_r * cos(*cached_th);
}

double synth_normal(uint64_t seed, uint64_t i) {
  uint64_t cp = UINT64_MAX;
  double r = 0.0, th = 0.0;
  return normal_at(seed, i, &cp, &r, &th);
}

/* kind: 1 = uint8, 2 = uint16, 3 = float32.  starts is [n_pulses][n_chan]. */
int synth_fill(int kind, void* out, int32_t n_chan, int64_t n_samp, int64_t row_stride,
               uint64_t seed, double mean, double sd, double lo, double hi,
               int32_t n_pulses, const int64_t* starts, const int64_t* widths,
               const double* amps) {
  if (!out || n_chan < 0 || n_samp < 0 || row_stride < n_samp) return -1;
  if (kind < 1 || kind > 3) return -1;
  if (n_pulses > 0 && (!starts || !widths || !amps)) return -1;
  int failed = 0;
#pragma omp parallel for schedule(static)
  for (int32_t c = 0; c < n_chan; ++c) {
    double* row = (double*)malloc((size_t)(n_samp > 0 ? n_samp : 1) * sizeof(double));
    if (!row) { failed = 1; continue; }
    uint64_t cp = UINT64_MAX;
    double r = 0.0, th = 0.0;
    uint64_t base = (uint64_t)c * (uint64_t)n_samp;
    for (int64_t t = 0; t < n_samp; ++t)
      row[t] = mean + sd * normal_at(seed, base + (uint64_t)t, &cp, &r, &th);
    for (int32_t p = 0; p < n_pulses; ++p) {
      int64_t s0 = starts[(int64_t)p * n_chan + c];
      for (int64_t j = 0; j < widths[p]; ++j) {
        int64_t t = s0 + j;
        if (t >= 0 && t < n_samp) row[t] += amps[p];
      }
    }
    if (kind == 3) {
      float* o = (float*)out + (int64_t)c * row_stride;
      for (int64_t t = 0; t < n_samp; ++t) o[t] = (float)row[t];
    } else {
      for (int64_t t = 0; t < n_samp; ++t) {
        double v = floor(row[t] + 0.5);
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        if (kind == 1)
          ((uint8_t*)out)[(int64_t)c * row_stride + t] = (uint8_t)v;
        else
          ((uint16_t*)out)[(int64_t)c * row_stride + t] = (uint16_t)v;
      }
    }
    free(row);
  }
  return failed ? -3 : 0;
}
