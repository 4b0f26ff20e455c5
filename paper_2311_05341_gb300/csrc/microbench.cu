// microbench.cu -- register-only kernels that measure the add-issue and
// shared-memory ceilings of the running GPU (declared in include/dd_bench.h).
// The dedispersion kernels are bound by these rates, not by HBM, so the
// benchmark reports achieved channel-adds against the rates measured here.
#include <cuda_runtime.h>

#include "dd.h"
#include "dd_bench.h"
#include "dd_internal.h"

namespace dd {
namespace {

constexpr int kAcc = 16;

__global__ void bench_iadd3(int64_t iters, uint32_t* sink) {
  uint32_t a[kAcc];
#pragma unroll
  for (int i = 0; i < kAcc; ++i) a[i] = threadIdx.x * 7u + i;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kAcc; ++i) a[i] = a[i] + a[(i + 5) % kAcc] + a[(i + 11) % kAcc];
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kAcc; ++i) s ^= a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void bench_iadd2(int64_t iters, uint32_t* sink) {
  uint32_t a[kAcc];
#pragma unroll
  for (int i = 0; i < kAcc; ++i) a[i] = threadIdx.x * 7u + i;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kAcc; ++i) a[i] = a[i] + a[(i + 5) % kAcc];
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kAcc; ++i) s ^= a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void bench_fadd(int64_t iters, uint32_t* sink) {
  float a[kAcc];
#pragma unroll
  for (int i = 0; i < kAcc; ++i) a[i] = 1e-30f * (threadIdx.x + i);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kAcc; ++i) a[i] = __fadd_rn(a[i], a[(i + 5) % kAcc]);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kAcc; ++i) s += a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = __float_as_uint(s);
}

__global__ void bench_fadd2(int64_t iters, uint32_t* sink) {
  unsigned long long a[kAcc];
#pragma unroll
  for (int i = 0; i < kAcc; ++i) {
    float lo = 1e-30f * (threadIdx.x + i), hi = 2e-30f * (threadIdx.x + i);
    a[i] = (static_cast<unsigned long long>(__float_as_uint(hi)) << 32) | __float_as_uint(lo);
  }
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kAcc; ++i) {
      unsigned long long r;
      asm volatile("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a[i]), "l"(a[(i + 5) % kAcc]));
      a[i] = r;
    }
  }
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < kAcc; ++i) s ^= a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = static_cast<uint32_t>(s ^ (s >> 32));
}

__global__ void bench_iadd3_imad(int64_t iters, uint32_t one, uint32_t* sink) {
  uint32_t a[kAcc];
#pragma unroll
  for (int i = 0; i < kAcc; ++i) a[i] = threadIdx.x * 7u + i;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kAcc; i += 2) {
      a[i] = a[i] + a[(i + 5) % kAcc] + a[(i + 11) % kAcc];
      uint32_t r;
      asm volatile("mad.lo.u32 %0, %1, %2, %3;"
                   : "=r"(r) : "r"(a[(i + 6) % kAcc]), "r"(one), "r"(a[i + 1]));
      a[i + 1] = r;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kAcc; ++i) s ^= a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void bench_lds128(int64_t iters, uint32_t* sink) {
  __shared__ uint4 buf[2048];  // 32 KiB
  for (int i = threadIdx.x; i < 2048; i += blockDim.x)
    buf[i] = make_uint4(i, i * 3u, i * 5u, i * 7u);
  __syncthreads();
  uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  uint32_t idx = threadIdx.x;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint4 v = buf[(idx + k * 32) & 2047];
      s0 ^= v.x; s1 ^= v.y; s2 ^= v.z; s3 ^= v.w;
    }
    idx += 256 + (s0 & 1);
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s0 ^ s1 ^ s2 ^ s3;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_bench_launch(int32_t kind, int32_t blocks, int32_t threads, int64_t iters,
                          uint32_t* d_sink, void* stream, double* ops_per_thread_iter) {
  if (!d_sink || !ops_per_thread_iter || blocks <= 0 || threads <= 0 || threads > 1024 ||
      iters < 0)
    return fail(DD_ERR_INVALID_ARG, "bad microbenchmark arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double ops = 0.0;
  switch (kind) {
    case DD_BENCH_IADD3: bench_iadd3<<<blocks, threads, 0, st>>>(iters, d_sink); ops = kAcc; break;
    case DD_BENCH_IADD2: bench_iadd2<<<blocks, threads, 0, st>>>(iters, d_sink); ops = kAcc; break;
    case DD_BENCH_FADD: bench_fadd<<<blocks, threads, 0, st>>>(iters, d_sink); ops = kAcc; break;
    case DD_BENCH_FADD2: bench_fadd2<<<blocks, threads, 0, st>>>(iters, d_sink); ops = kAcc; break;
    case DD_BENCH_IADD3_IMAD:
      bench_iadd3_imad<<<blocks, threads, 0, st>>>(iters, 1u, d_sink);
      ops = kAcc;
      break;
    case DD_BENCH_LDS128: bench_lds128<<<blocks, threads, 0, st>>>(iters, d_sink); ops = 8; break;
    default: return fail(DD_ERR_INVALID_ARG, "unknown microbenchmark kind");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "dd_bench_launch");
  *ops_per_thread_iter = ops;
  return DD_OK;
}

dd_status dd_bench_device(int32_t* sm_count, int32_t* max_clock_khz) {
  if (!sm_count || !max_clock_khz) return fail(DD_ERR_INVALID_ARG, "NULL output");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  int sms = 0, clk = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  *sm_count = sms;
  *max_clock_khz = clk;
  return DD_OK;
}

}  // extern "C"
