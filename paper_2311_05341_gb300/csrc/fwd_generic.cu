// fwd_generic.cu -- shared-memory forward dedispersion kernel for every input
// dtype (uint8, uint16, float32, packed 4-bit) and every time bin.
//
// Eq. 3 / Algorithm 1: Y[d][t] = sum_c X_b[c][t + s(c, d)].  The output
// (DM, t) plane is cut into CTA tiles of kGenDmPerCta DMs x kGenSampPerCta
// samples (the paper's D_dm x D_t partition, Sec. 4).  For each chunk of
// channels the CTA stages, per channel, the window
//   X_b[c][t0 + s(c, d_first) + k],  k < kGenSampPerCta + span,
// into shared memory (decimation by the range's bin fused into the staging
// load, Sec. 5.3), and every thread adds, for each of its DMs, the window
// entries at the DM's offset s(c, d) - s(c, d_first) into register
// accumulators (the B_loc / S_loc structure of the paper's Algorithm 3).
// This kernel serves all dtypes and plans; uint8 plans with bin 1 have a
// faster dedicated kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include "dd_internal.h"

namespace dd {

namespace {

// Raw sample i of a channel row: 4-bit rows (NIB) hold two samples per byte,
// the earlier in the low nibble.
template <typename TIn, typename TAcc, bool NIB>
__device__ __forceinline__ TAcc raw_sample(const TIn* row, int64_t i) {
  if constexpr (NIB) return static_cast<TAcc>((row[i >> 1] >> (4 * (i & 1))) & 15);
  else return static_cast<TAcc>(row[i]);
}

template <typename TIn, typename TAcc, bool NIB>
__global__ void __launch_bounds__(256)
fwd_generic_kernel(const TIn* __restrict__ x, int64_t stride, int32_t n_chan, int32_t bin,
                   int64_t n_dec, const int32_t* __restrict__ shifts, int32_t n_dm,
                   int32_t n_dm_blocks, int64_t n_out, int64_t tile0, int64_t t_end,
                   int32_t win, int32_t chunk, TAcc* __restrict__ out) {
  extern __shared__ unsigned char smem_raw[];
  TAcc* win_buf = reinterpret_cast<TAcc*>(smem_raw);              // [chunk][win]
  int32_t* base_buf = reinterpret_cast<int32_t*>(win_buf + chunk * win);  // [chunk]

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t tile = blockIdx.x / n_dm_blocks + tile0;
  const int32_t dblk = blockIdx.x % n_dm_blocks;
  const int32_t d_first = dblk * kGenDmPerCta;
  const int64_t t0 = tile * kGenSampPerCta;

  int32_t my_d[kGenDmPerThread];
#pragma unroll
  for (int i = 0; i < kGenDmPerThread; ++i)
    my_d[i] = min(d_first + ty + 8 * i, n_dm - 1);

  TAcc acc[kGenDmPerThread][kGenSampPerThread];
#pragma unroll
  for (int i = 0; i < kGenDmPerThread; ++i)
#pragma unroll
    for (int k = 0; k < kGenSampPerThread; ++k) acc[i][k] = TAcc(0);

  for (int32_t c0 = 0; c0 < n_chan; c0 += chunk) {
    const int32_t nc = min(chunk, n_chan - c0);
    __syncthreads();
    // Stage: warp ty loads channels ty, ty+8, ... of the chunk, lanes along time.
    for (int32_t cc = ty; cc < nc; cc += 8) {
      const int32_t c = c0 + cc;
      const int32_t base = shifts[static_cast<int64_t>(d_first) * n_chan + c];
      if (tx == 0) base_buf[cc] = base;
      const TIn* row = x + static_cast<int64_t>(c) * (NIB ? stride / 2 : stride);
      for (int32_t k = tx; k < win; k += 32) {
        const int64_t u = t0 + base + k;  // decimated sample index
        TAcc v = TAcc(0);
        if (u < n_dec) {
          const int64_t raw = u * bin;
          for (int32_t j = 0; j < bin; ++j) v += raw_sample<TIn, TAcc, NIB>(row, raw + j);
        }
        win_buf[cc * win + k] = v;
      }
    }
    __syncthreads();
    for (int32_t cc = 0; cc < nc; ++cc) {
      const int32_t c = c0 + cc;
      const int32_t base = base_buf[cc];
      const TAcc* w = win_buf + cc * win + tx;
#pragma unroll
      for (int i = 0; i < kGenDmPerThread; ++i) {
        const int32_t delta = shifts[static_cast<int64_t>(my_d[i]) * n_chan + c] - base;
#pragma unroll
        for (int k = 0; k < kGenSampPerThread; ++k) acc[i][k] += w[delta + 32 * k];
      }
    }
  }

#pragma unroll
  for (int i = 0; i < kGenDmPerThread; ++i) {
    const int32_t d = d_first + ty + 8 * i;
    if (d >= n_dm) continue;
    TAcc* orow = out + static_cast<int64_t>(d) * n_out;
#pragma unroll
    for (int k = 0; k < kGenSampPerThread; ++k) {
      const int64_t t = t0 + tx + 32 * k;
      if (t < t_end) orow[t] = acc[i][k];
    }
  }
}

template <typename TIn, typename TAcc, bool NIB = false>
int launch_typed(const dd_plan_s* p, const RangePlan& rp, const void* d_in, int64_t stride,
                 int64_t n_samp, int64_t n_out, void* d_out, int64_t t_begin, int64_t t_end,
                 cudaStream_t st) {
  if (t_begin % kGenSampPerCta != 0 || t_begin < 0 || t_end > n_out || t_end <= t_begin)
    return static_cast<int>(cudaErrorInvalidValue);
  const int32_t win = kGenSampPerCta + rp.gen_span;
  const size_t per_chan = static_cast<size_t>(win) * sizeof(TAcc) + sizeof(int32_t);
  int32_t chunk = static_cast<int32_t>(std::min<size_t>(32, (96 * 1024) / per_chan));
  if (chunk < 1) return static_cast<int>(cudaErrorInvalidConfiguration);
  chunk = std::min(chunk, p->n_chan);
  const size_t smem = per_chan * chunk + 16;
  auto kern = fwd_generic_kernel<TIn, TAcc, NIB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  const int64_t tile0 = t_begin / kGenSampPerCta;
  const int64_t tiles = (t_end + kGenSampPerCta - 1) / kGenSampPerCta - tile0;
  const int64_t grid = tiles * rp.gen_n_blocks;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  const int32_t* shifts = reinterpret_cast<const int32_t*>(
      static_cast<const unsigned char*>(p->d_ws) + rp.off_shifts);
  kern<<<static_cast<unsigned>(grid), dim3(32, 8), smem, st>>>(
      static_cast<const TIn*>(d_in), stride, p->n_chan, rp.r.bin, n_samp / rp.r.bin, shifts,
      static_cast<int32_t>(rp.n_dm), rp.gen_n_blocks, n_out, tile0, t_end, win, chunk,
      static_cast<TAcc*>(d_out));
  return static_cast<int>(cudaGetLastError());
}

}  // namespace

int launch_forward_generic(const dd_plan_s* p, const RangePlan& rp, const void* d_in,
                           int64_t stride, int64_t n_samp, int64_t n_out, void* d_out,
                           int64_t t_begin, int64_t t_end, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (p->dtype) {
    case DD_U8:
      return launch_typed<uint8_t, int32_t>(p, rp, d_in, stride, n_samp, n_out, d_out, t_begin,
                                            t_end, st);
    case DD_U16:
      return launch_typed<uint16_t, int32_t>(p, rp, d_in, stride, n_samp, n_out, d_out, t_begin,
                                             t_end, st);
    case DD_U4:
      return launch_typed<uint8_t, int32_t, true>(p, rp, d_in, stride, n_samp, n_out, d_out,
                                                  t_begin, t_end, st);
    case DD_F32:
      return launch_typed<float, float>(p, rp, d_in, stride, n_samp, n_out, d_out, t_begin, t_end,
                                        st);
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

}  // namespace dd
