/*
 * dd_cpu_tiled.c -- a tiled CPU implementation of the direct dedispersion
 * transform (Eq. 3), after the paper's CPU code (Sec. 3, Algorithm 2): the
 * (DM, time) plane is cut into tiles of DT_DM DMs x DT_T samples processed in
 * parallel (OpenMP over both tile indices), and within a tile every channel's
 * shifted row segment is added into per-DM accumulator vectors that stay in
 * cache.  It is a stronger CPU baseline than the plain oracle for the
 * benchmark; it is not used by the GPU library and is not the parity
 * authority (tests compare it with the oracle).
 *
 * Shifts are taken as a precomputed int32 table [n_dm][n_chan] (the caller
 * builds it with the planner), time bin 1, raw sums: Y[d][t] = sum_c X[c][t +
 * s(c, d)] for t < n_out.  uint8 / uint16 inputs sum into int32, float32 into
 * float.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DT_DM 16
#define DT_T 2048

int dd_cpu_tiled(int dtype, const void* x, int32_t n_chan, int64_t row_stride,
                 const int32_t* shifts, int32_t n_dm, int64_t n_out, void* out) {
  if (!x || !shifts || !out || n_chan <= 0 || n_dm <= 0 || n_out <= 0) return -1;
  if (dtype < 1 || dtype > 3) return -1;
  const int64_t n_tt = (n_out + DT_T - 1) / DT_T;
  const int64_t n_td = (n_dm + DT_DM - 1) / DT_DM;
  int failed = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int64_t td = 0; td < n_td; ++td) {
    for (int64_t tt = 0; tt < n_tt; ++tt) {
      const int32_t d0 = (int32_t)(td * DT_DM);
      const int32_t nd = (n_dm - d0) < DT_DM ? (n_dm - d0) : DT_DM;
      const int64_t t0 = tt * DT_T;
      const int64_t nt = (n_out - t0) < DT_T ? (n_out - t0) : DT_T;
      if (dtype == 3) {
        float* acc = (float*)calloc((size_t)DT_DM * DT_T, sizeof(float));
        if (!acc) { failed = 1; continue; }
        for (int32_t c = 0; c < n_chan; ++c) {
          const float* row = (const float*)x + (int64_t)c * row_stride + t0;
          for (int32_t i = 0; i < nd; ++i) {
            const float* src = row + shifts[(int64_t)(d0 + i) * n_chan + c];
            float* a = acc + (int64_t)i * DT_T;
            for (int64_t t = 0; t < nt; ++t) a[t] += src[t];
          }
        }
        for (int32_t i = 0; i < nd; ++i)
          memcpy((float*)out + (int64_t)(d0 + i) * n_out + t0, acc + (int64_t)i * DT_T,
                 (size_t)nt * sizeof(float));
        free(acc);
      } else {
        int32_t* acc = (int32_t*)calloc((size_t)DT_DM * DT_T, sizeof(int32_t));
        if (!acc) { failed = 1; continue; }
        for (int32_t c = 0; c < n_chan; ++c) {
          for (int32_t i = 0; i < nd; ++i) {
            const int64_t off = (int64_t)c * row_stride + t0 + shifts[(int64_t)(d0 + i) * n_chan + c];
            int32_t* a = acc + (int64_t)i * DT_T;
            if (dtype == 1) {
              const uint8_t* src = (const uint8_t*)x + off;
              for (int64_t t = 0; t < nt; ++t) a[t] += src[t];
            } else {
              const uint16_t* src = (const uint16_t*)x + off;
              for (int64_t t = 0; t < nt; ++t) a[t] += src[t];
            }
          }
        }
        for (int32_t i = 0; i < nd; ++i)
          memcpy((int32_t*)out + (int64_t)(d0 + i) * n_out + t0, acc + (int64_t)i * DT_T,
                 (size_t)nt * sizeof(int32_t));
        free(acc);
      }
    }
  }
  return failed ? -3 : 0;
}
