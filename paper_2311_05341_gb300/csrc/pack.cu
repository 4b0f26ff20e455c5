// pack.cu -- the packed copy of a uint8 (or 4-bit) filterbank read by the
// kU8P pattern tiles (uint16: the copy widened to 32-bit words, kU16P; float32:
// 64-bit words of two floats, kF32P): word t of channel c holds samples t and t + pair in its 16-bit halves,
//   W[c][t] = X[c][t] | X[c][t + pair] << 16   (0 where an index reaches n_samp),
// so the tiles stage window words without unpacking.  HBM-bound: reads the
// input twice (the second read mostly from L2) and writes four bytes per sample.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace dd {

namespace {

constexpr int kPackPerThread = 16;  // samples per thread: one 16-byte load per half

__device__ __forceinline__ uint32_t sample_at(const uint8_t* row, int64_t t, int64_t n) {
  return t < n ? row[t] : 0u;
}

__global__ void __launch_bounds__(256) pack_pairs_kernel(const uint8_t* __restrict__ in,
                                                         int64_t in_stride, int64_t n_samp,
                                                         uint32_t* __restrict__ out,
                                                         int64_t out_stride, int32_t pair,
                                                         int64_t chunks_per_row, int32_t n_chan,
                                                         int64_t t_begin, int64_t t_end,
                                                         int64_t origin) {
  const int64_t gid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t c = gid / chunks_per_row;
  const int64_t t = t_begin + (gid - c * chunks_per_row) * kPackPerThread;
  if (c >= n_chan || t >= t_end) return;  // the last block's spare threads
  const uint8_t* row = in + c * in_stride;
  uint32_t* dst = out + c * out_stride + (t - origin);
  uint32_t w[kPackPerThread];
  if (t + pair + kPackPerThread <= n_samp) {
    // Both halves inside the row: two aligned 16-byte loads (t, pair and the
    // row stride are multiples of 16).
    const uint4 a = *reinterpret_cast<const uint4*>(row + t);
    const uint4 b = *reinterpret_cast<const uint4*>(row + t + pair);
    const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      w[4 * k + 0] = __byte_perm(av[k], bv[k], 0x4440) & 0x00ff00ffu;
      w[4 * k + 1] = __byte_perm(av[k], bv[k], 0x4541) & 0x00ff00ffu;
      w[4 * k + 2] = __byte_perm(av[k], bv[k], 0x4642) & 0x00ff00ffu;
      w[4 * k + 3] = __byte_perm(av[k], bv[k], 0x4743) & 0x00ff00ffu;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kPackPerThread; ++k)
      w[k] = sample_at(row, t + k, n_samp) | sample_at(row, t + k + pair, n_samp) << 16;
  }
  // t_end is a multiple of 4 words; the range's last chunk may be partial.
#pragma unroll
  for (int k = 0; k < kPackPerThread; k += 4)
    if (t + k < t_end)
      *reinterpret_cast<uint4*>(dst + k) = make_uint4(w[k], w[k + 1], w[k + 2], w[k + 3]);
}

// The same packed words from 4-bit input (two samples per byte, the earlier
// in the low nibble; in_stride in bytes).
__device__ __forceinline__ uint32_t nibble_at(const uint8_t* row, int64_t t, int64_t n) {
  return t < n ? (row[t >> 1] >> (4 * (t & 1))) & 0xfu : 0u;
}

__global__ void __launch_bounds__(256) pack_pairs4_kernel(const uint8_t* __restrict__ in,
                                                          int64_t in_stride, int64_t n_samp,
                                                          uint32_t* __restrict__ out,
                                                          int64_t out_stride, int32_t pair,
                                                          int64_t chunks_per_row, int32_t n_chan,
                                                          int64_t t_begin, int64_t t_end, int64_t origin) {
  const int64_t gid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t c = gid / chunks_per_row;
  const int64_t t = t_begin + (gid - c * chunks_per_row) * kPackPerThread;
  if (c >= n_chan || t >= t_end) return;  // the last block's spare threads
  const uint8_t* row = in + c * in_stride;
  uint32_t* dst = out + c * out_stride + (t - origin);
  uint32_t w[kPackPerThread];
  if (t + pair + kPackPerThread <= n_samp) {
    // Both halves inside the row: two aligned 8-byte loads (t, pair and the
    // row stride in samples are multiples of 16).
    const uint2 a = *reinterpret_cast<const uint2*>(row + (t >> 1));
    const uint2 b = *reinterpret_cast<const uint2*>(row + ((t + pair) >> 1));
    const uint32_t av[2] = {a.x, a.y}, bv[2] = {b.x, b.y};
#pragma unroll
    for (int k = 0; k < kPackPerThread; ++k) {
      const int sh = 4 * (k & 7);
      w[k] = ((av[k >> 3] >> sh) & 0xfu) | ((bv[k >> 3] >> sh) & 0xfu) << 16;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kPackPerThread; ++k)
      w[k] = nibble_at(row, t + k, n_samp) | nibble_at(row, t + k + pair, n_samp) << 16;
  }
#pragma unroll
  for (int k = 0; k < kPackPerThread; k += 4)
    if (t + k < t_end)
      *reinterpret_cast<uint4*>(dst + k) = make_uint4(w[k], w[k + 1], w[k + 2], w[k + 3]);
}

// uint16 input widened to one sample per 32-bit word (pair unused).
__global__ void __launch_bounds__(256) widen16_kernel(const uint8_t* __restrict__ in,
                                                      int64_t in_stride, int64_t n_samp,
                                                      uint32_t* __restrict__ out,
                                                      int64_t out_stride, int64_t chunks_per_row,
                                                      int32_t n_chan, int64_t t_begin,
                                                      int64_t t_end, int64_t origin) {
  const int64_t gid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t c = gid / chunks_per_row;
  const int64_t t = t_begin + (gid - c * chunks_per_row) * kPackPerThread;
  if (c >= n_chan || t >= t_end) return;  // the last block's spare threads
  const uint16_t* row = reinterpret_cast<const uint16_t*>(in + c * in_stride);
  uint32_t* dst = out + c * out_stride + (t - origin);
  uint32_t w[kPackPerThread];
  if (t + kPackPerThread <= n_samp) {
    // Two aligned 16-byte loads (t is a multiple of 16, rows 16-byte aligned).
    const uint4 a = *reinterpret_cast<const uint4*>(row + t);
    const uint4 b = *reinterpret_cast<const uint4*>(row + t + 8);
    const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      w[2 * k] = v[k] & 0xffffu;
      w[2 * k + 1] = v[k] >> 16;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kPackPerThread; ++k) w[k] = t + k < n_samp ? row[t + k] : 0u;
  }
#pragma unroll
  for (int k = 0; k < kPackPerThread; k += 4)
    if (t + k < t_end)
      *reinterpret_cast<uint4*>(dst + k) = make_uint4(w[k], w[k + 1], w[k + 2], w[k + 3]);
}

// float32 pairs: 64-bit word t = (X[t], X[t + pair]) as two floats (0 past
// n_samp); out_stride counts 64-bit words.  Each thread writes 4 words.
__global__ void __launch_bounds__(256) pack_f32_pairs_kernel(const float* __restrict__ in,
                                                             int64_t in_stride, int64_t n_samp,
                                                             float2* __restrict__ out,
                                                             int64_t out_stride, int32_t pair,
                                                             int64_t chunks_per_row,
                                                             int32_t n_chan, int64_t t_begin,
                                                             int64_t t_end, int64_t origin) {
  const int64_t gid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t c = gid / chunks_per_row;
  const int64_t t = t_begin + (gid - c * chunks_per_row) * 4;
  if (c >= n_chan || t >= t_end) return;  // the last block's spare threads
  const float* row = in + c * in_stride;
  float2* dst = out + c * out_stride + (t - origin);
  float a[4], b[4];
  if (t + pair + 4 <= n_samp) {
    // Both halves inside the row: two aligned 16-byte loads (t, pair and the
    // row stride are multiples of 4 floats).
    const float4 va = *reinterpret_cast<const float4*>(row + t);
    const float4 vb = *reinterpret_cast<const float4*>(row + t + pair);
    a[0] = va.x; a[1] = va.y; a[2] = va.z; a[3] = va.w;
    b[0] = vb.x; b[1] = vb.y; b[2] = vb.z; b[3] = vb.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = t + k < n_samp ? row[t + k] : 0.f;
      b[k] = t + k + pair < n_samp ? row[t + k + pair] : 0.f;
    }
  }
  // t_end is a multiple of 4 words, so a thread's 4 words are all in range.
  reinterpret_cast<float4*>(dst)[0] = make_float4(a[0], b[0], a[1], b[1]);
  reinterpret_cast<float4*>(dst)[1] = make_float4(a[2], b[2], a[3], b[3]);
}

// uint8 decimated by a time bin b (2, 4 or 8) into the packed pair words:
// word t = D[t] | D[t + pair] << 16 with D[t] = sum_{j < b} X[b t + j], the
// decimated sample (Sec. 5.3's binning), for t < n_dec = floor(n_samp / b), 0
// past it.  Each thread writes 4 words (out_stride and the output length are
// multiples of 4).
template <int B>
__device__ __forceinline__ uint32_t dec_at(const uint8_t* row, int64_t t, int64_t n_dec) {
  if (t >= n_dec) return 0u;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < B; ++j) s += row[B * t + j];
  return s;
}

template <int B>
__device__ __forceinline__ void dec4(const uint8_t* row, int64_t t, uint32_t (&d)[4]) {
  // 4 decimated samples from 4 B aligned bytes (B = 2: 8, 4: 16, 8: 32 bytes).
  if constexpr (B == 2) {
    const uint2 a = *reinterpret_cast<const uint2*>(row + 2 * t);
    const uint32_t s0 = (a.x & 0x00ff00ffu) + ((a.x >> 8) & 0x00ff00ffu);
    const uint32_t s1 = (a.y & 0x00ff00ffu) + ((a.y >> 8) & 0x00ff00ffu);
    d[0] = s0 & 0xffffu; d[1] = s0 >> 16; d[2] = s1 & 0xffffu; d[3] = s1 >> 16;
  } else if constexpr (B == 4) {
    const uint4 a = *reinterpret_cast<const uint4*>(row + 4 * t);
    d[0] = __dp4a(a.x, 0x01010101u, 0u); d[1] = __dp4a(a.y, 0x01010101u, 0u);
    d[2] = __dp4a(a.z, 0x01010101u, 0u); d[3] = __dp4a(a.w, 0x01010101u, 0u);
  } else {
    const uint4 a = *reinterpret_cast<const uint4*>(row + 8 * t);
    const uint4 b = *reinterpret_cast<const uint4*>(row + 8 * t + 16);
    d[0] = __dp4a(a.y, 0x01010101u, __dp4a(a.x, 0x01010101u, 0u));
    d[1] = __dp4a(a.w, 0x01010101u, __dp4a(a.z, 0x01010101u, 0u));
    d[2] = __dp4a(b.y, 0x01010101u, __dp4a(b.x, 0x01010101u, 0u));
    d[3] = __dp4a(b.w, 0x01010101u, __dp4a(b.z, 0x01010101u, 0u));
  }
}

template <int B>
__global__ void __launch_bounds__(256) pack_pairs_binned_kernel(
    const uint8_t* __restrict__ in, int64_t in_stride, int64_t n_samp, uint32_t* __restrict__ out,
    int64_t out_stride, int32_t pair, int64_t chunks_per_row, int32_t n_chan) {
  const int64_t gid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t c = gid / chunks_per_row;
  const int64_t t = (gid - c * chunks_per_row) * 4;
  if (c >= n_chan) return;  // the last block's spare threads
  const uint8_t* row = in + c * in_stride;
  const int64_t n_dec = n_samp / B;
  uint32_t lo[4], hi[4];
  if (t + pair + 4 <= n_dec) {
    dec4<B>(row, t, lo);
    dec4<B>(row, t + pair, hi);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      lo[k] = dec_at<B>(row, t + k, n_dec);
      hi[k] = dec_at<B>(row, t + k + pair, n_dec);
    }
  }
  *reinterpret_cast<uint4*>(out + c * out_stride + t) =
      make_uint4(lo[0] | hi[0] << 16, lo[1] | hi[1] << 16, lo[2] | hi[2] << 16, lo[3] | hi[3] << 16);
}

}  // namespace

int launch_pack_pairs_binned(const void* d_in, int64_t in_stride, int32_t n_chan, int64_t n_samp,
                             int32_t bin, void* d_out, int64_t out_stride, int32_t pair,
                             void* stream) {
  if (n_chan <= 0 || n_samp <= 0) return 0;
  if (pair % 16 != 0 || in_stride % 16 != 0 || out_stride % 4 != 0 ||
      out_stride < n_samp / bin || (bin != 2 && bin != 4 && bin != 8))
    return static_cast<int>(cudaErrorInvalidValue);
  const int64_t chunks = out_stride / 4;
  const int64_t blocks = (chunks * n_chan + 255) / 256;
  if (blocks > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  const auto* in = static_cast<const uint8_t*>(d_in);
  auto* out = static_cast<uint32_t*>(d_out);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned g = static_cast<unsigned>(blocks);
  if (bin == 2)
    pack_pairs_binned_kernel<2><<<g, 256, 0, st>>>(in, in_stride, n_samp, out, out_stride, pair,
                                                   chunks, n_chan);
  else if (bin == 4)
    pack_pairs_binned_kernel<4><<<g, 256, 0, st>>>(in, in_stride, n_samp, out, out_stride, pair,
                                                   chunks, n_chan);
  else
    pack_pairs_binned_kernel<8><<<g, 256, 0, st>>>(in, in_stride, n_samp, out, out_stride, pair,
                                                   chunks, n_chan);
  return static_cast<int>(cudaGetLastError());
}

int launch_pack_pairs(const void* d_in, int64_t in_stride, int32_t n_chan, int64_t n_samp,
                      void* d_out, int64_t out_stride, int32_t pair, int64_t t_begin,
                      int64_t t_end, PackSource src, void* stream, int64_t out_origin) {
  if (n_chan <= 0 || n_samp <= 0 || t_end <= t_begin) return 0;
  if (pair % 16 != 0 || in_stride % 16 != 0 || out_stride % 4 != 0 || out_origin < 0 ||
      out_origin % 16 != 0 || t_begin % 16 != 0 || t_begin < out_origin || t_end % 4 != 0 ||
      t_end > out_origin + out_stride)
    return static_cast<int>(cudaErrorInvalidValue);
  if (src == PackSource::kF32) {
    const int64_t chunks = (t_end - t_begin) / 4;
    const int64_t blocks = (chunks * n_chan + 255) / 256;
    if (blocks > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
    pack_f32_pairs_kernel<<<static_cast<unsigned>(blocks), 256, 0,
                            static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float*>(d_in), in_stride / 4, n_samp, static_cast<float2*>(d_out),
        out_stride, pair, chunks, n_chan, t_begin, t_end, out_origin);
    return static_cast<int>(cudaGetLastError());
  }
  const int64_t chunks = (t_end - t_begin + kPackPerThread - 1) / kPackPerThread;
  const int64_t threads = chunks * n_chan;
  const int64_t blocks = (threads + 255) / 256;
  if (blocks > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  const auto* in = static_cast<const uint8_t*>(d_in);
  auto* out = static_cast<uint32_t*>(d_out);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (src == PackSource::kU16)
    widen16_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        in, in_stride, n_samp, out, out_stride, chunks, n_chan, t_begin, t_end, out_origin);
  else if (src == PackSource::kU4)
    pack_pairs4_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        in, in_stride, n_samp, out, out_stride, pair, chunks, n_chan, t_begin, t_end, out_origin);
  else
    pack_pairs_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        in, in_stride, n_samp, out, out_stride, pair, chunks, n_chan, t_begin, t_end, out_origin);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace dd
