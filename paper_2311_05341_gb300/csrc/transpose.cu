// transpose.cu -- front end: time-major filterbank samples (the order a
// receiver or a SIGPROC file delivers, X_tm[t][c]) to the channel-major rows
// the dedispersion kernels read (X[c][t]).
//
// Work is in 32-bit words of R = 4 / sample-bytes samples.  A CTA moves a tile
// of 32R times x 32R channels = 32 x 32 words: it loads the tile's 32R time
// rows with coalesced 128-byte reads into shared memory (column index XOR the
// row's word-row, so both phases are free of bank conflicts), then each thread
// takes R x R sample blocks, transposes them in registers (byte or half-word
// permutes) and writes R words along time, 128 contiguous bytes per warp and
// channel row.  Only samples with t in [t_begin, t_end) and c < n_chan are
// written; words that straddle t_end are written sample by sample.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace dd {

namespace {

constexpr int kTileWords = 32;

// Sample j (0..R-1) of a word of R samples.
template <int R>
__device__ __forceinline__ uint32_t sample_of(uint32_t w, int j) {
  if constexpr (R == 4) return (w >> (8 * j)) & 0xffu;
  else if constexpr (R == 2) return (w >> (16 * j)) & 0xffffu;
  else return w;
}

// Transpose of an R x R block held as R words (word r = time r, samples =
// channels): out[j] = channel j, samples = times.
template <int R>
__device__ __forceinline__ void block_transpose(const uint32_t (&in)[R], uint32_t (&out)[R]) {
  if constexpr (R == 4) {
    // Bytes: in[r] = (c0 c1 c2 c3) at time r.
    const uint32_t a = __byte_perm(in[0], in[1], 0x5140);  // t0c0 t1c0 t0c1 t1c1
    const uint32_t b = __byte_perm(in[2], in[3], 0x5140);  // t2c0 t3c0 t2c1 t3c1
    const uint32_t c = __byte_perm(in[0], in[1], 0x7362);  // t0c2 t1c2 t0c3 t1c3
    const uint32_t d = __byte_perm(in[2], in[3], 0x7362);  // t2c2 t3c2 t2c3 t3c3
    out[0] = __byte_perm(a, b, 0x5410);
    out[1] = __byte_perm(a, b, 0x7632);
    out[2] = __byte_perm(c, d, 0x5410);
    out[3] = __byte_perm(c, d, 0x7632);
  } else if constexpr (R == 2) {
    out[0] = __byte_perm(in[0], in[1], 0x5410);
    out[1] = __byte_perm(in[0], in[1], 0x7632);
  } else {
    out[0] = in[0];
  }
}

template <int E>
__global__ void __launch_bounds__(256) transpose_kernel(const uint8_t* __restrict__ in,
                                                        int64_t in_stride_bytes, int32_t n_chan,
                                                        uint8_t* __restrict__ out,
                                                        int64_t out_stride_bytes,
                                                        int64_t t_begin, int64_t t_end,
                                                        int32_t chan_tiles) {
  constexpr int R = 4 / E;
  constexpr int kRows = kTileWords * R;  // times (and channels) per tile
  __shared__ uint32_t tile[kRows][kTileWords];
  const int tid = threadIdx.x;
  const int64_t t0 = t_begin + static_cast<int64_t>(blockIdx.x / chan_tiles) * kRows;
  const int32_t c0 = (blockIdx.x % chan_tiles) * kRows;
  const int64_t in_words = in_stride_bytes / 4;  // words per time row (rows are 16-byte aligned)
  const int32_t cw0 = c0 / R;                    // first channel word of the tile

  // Load: warp-wide 128-byte row reads; row i holds time t0 + i.
  for (int i = tid / kTileWords; i < kRows; i += 256 / kTileWords) {
    const int col = tid % kTileWords;
    const int64_t t = t0 + i;
    uint32_t v = 0;
    if (t < t_end && cw0 + col < in_words)
      v = __ldg(reinterpret_cast<const uint32_t*>(in + t * in_stride_bytes) + cw0 + col);
    tile[i][col ^ ((i / R) % kTileWords)] = v;
  }
  __syncthreads();

  // Blocks: thread takes word-row bt (times t0 + R bt ..) of word-column bc.
  for (int k = tid; k < kTileWords * kTileWords; k += 256) {
    const int bt = k % kTileWords, bc = k / kTileWords;
    uint32_t w[R], o[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = tile[R * bt + r][bc ^ bt];
    block_transpose<R>(w, o);
    const int64_t t = t0 + static_cast<int64_t>(R) * bt;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int32_t c = c0 + R * bc + j;
      if (c >= n_chan || t >= t_end) continue;
      uint8_t* row = out + static_cast<int64_t>(c) * out_stride_bytes;
      if (t + R <= t_end) {
        *reinterpret_cast<uint32_t*>(row + t * E) = o[j];
      } else {
        for (int s = 0; s < R && t + s < t_end; ++s) {
          const uint32_t v = sample_of<R>(o[j], s);
          if constexpr (E == 1) row[t + s] = static_cast<uint8_t>(v);
          else if constexpr (E == 2) reinterpret_cast<uint16_t*>(row)[t + s] = static_cast<uint16_t>(v);
          else reinterpret_cast<uint32_t*>(row)[t + s] = v;
        }
      }
    }
  }
}

}  // namespace

int launch_transpose(int elem_bytes, const void* d_in, int64_t in_row_stride, int32_t n_chan,
                     void* d_out, int64_t out_row_stride, int64_t t_begin, int64_t t_end,
                     void* stream) {
  if (t_end <= t_begin) return 0;
  const int R = 4 / elem_bytes;
  const int rows = kTileWords * R;
  const int32_t chan_tiles = (n_chan + rows - 1) / rows;
  const int64_t time_tiles = (t_end - t_begin + rows - 1) / rows;
  const int64_t grid = time_tiles * chan_tiles;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const auto* in = static_cast<const uint8_t*>(d_in);
  auto* out = static_cast<uint8_t*>(d_out);
  const int64_t isb = in_row_stride * elem_bytes, osb = out_row_stride * elem_bytes;
  const unsigned g = static_cast<unsigned>(grid);
  switch (elem_bytes) {
    case 1: transpose_kernel<1><<<g, 256, 0, st>>>(in, isb, n_chan, out, osb, t_begin, t_end, chan_tiles); break;
    case 2: transpose_kernel<2><<<g, 256, 0, st>>>(in, isb, n_chan, out, osb, t_begin, t_end, chan_tiles); break;
    case 4: transpose_kernel<4><<<g, 256, 0, st>>>(in, isb, n_chan, out, osb, t_begin, t_end, chan_tiles); break;
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
  return static_cast<int>(cudaGetLastError());
}

}  // namespace dd
