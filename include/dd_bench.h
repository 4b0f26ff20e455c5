/*
 * dd_bench.h -- register-only microbenchmarks that measure the add-issue
 * roofline of the GPU the library runs on.
 *
 * Dedispersion with data reuse is bound by how fast the SM issues adds
 * (Sec. 2 counts one add per channel per output; with reuse the arithmetic
 * intensity far exceeds the HBM ridge point).  The paper's shared-memory
 * bandwidth formula (Eq. 8) gives the second ceiling; these kernels measure
 * both, plus the float add rate, under the clocks of the run, so that the
 * benchmark can report achieved adds as a fraction of a measured peak.
 *
 * Each kernel runs `iters` iterations of an unrolled body on blocks x threads
 * threads with no global memory traffic except one store per thread into
 * d_sink (device, blocks*threads uint32, caller-owned).  *ops_per_thread_iter
 * receives the number of counted operations per thread per iteration:
 *   DD_BENCH_IADD3      3-input 32-bit integer adds (counted as 1 op each)
 *   DD_BENCH_IADD2      2-input 32-bit integer adds
 *   DD_BENCH_FADD       float32 adds
 *   DD_BENCH_FADD2      packed float32x2 adds (add.rn.f32x2; counted as 1 op)
 *   DD_BENCH_IADD3_IMAD alternating 3-input adds and integer multiply-adds
 *                       used as adds (counted as 1 op each)
 *   DD_BENCH_LDS128     16-byte shared-memory loads (counted as 1 op = 16 bytes)
 * Time the launch with CUDA events on `stream`.
 */
#ifndef DD_BENCH_H
#define DD_BENCH_H

#include <stdint.h>

#include "dd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DD_BENCH_IADD3 = 1,
  DD_BENCH_IADD2 = 2,
  DD_BENCH_FADD = 3,
  DD_BENCH_FADD2 = 4,
  DD_BENCH_IADD3_IMAD = 5,
  DD_BENCH_LDS128 = 6
} dd_bench_kind;

dd_status dd_bench_launch(int32_t kind, int32_t blocks, int32_t threads, int64_t iters,
                          uint32_t* d_sink, void* stream, double* ops_per_thread_iter);

/* Number of SMs and the maximum SM clock (kHz) of the current device. */
dd_status dd_bench_device(int32_t* sm_count, int32_t* max_clock_khz);

#ifdef __cplusplus
}
#endif

#endif /* DD_BENCH_H */
