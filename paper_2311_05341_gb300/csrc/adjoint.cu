// adjoint.cu -- transpose of the forward transform for float32 plans
// (re-dispersion), written as a gather so that no atomics are needed:
//
//   xbar[c][t] = sum_r sum_d ybar_r[d][floor(t / b_r) - s_r(c, d)]
//
// over the terms with 0 <= floor(t/b_r) - s_r(c, d) < n_out_r.  Every input
// sample X[c][t] enters output Y_r[d][floor(t/b_r) - s_r(c,d)] with weight 1
// (Eq. 3 with time binning), so this is exactly the derivative of Eq. 3 with
// respect to X.  The paper has no adjoint; this mirrors its forward tiling with
// the roles of channel and DM swapped: a CTA owns 64 channels x 256 raw
// samples (8 warps x 8 channels, lane l: samples l + 32 k), and for each chunk
// of DMs it stages the needed window of each DM's output row in shared memory
// once for all 64 channels, then every thread gathers from it at each of its
// channels' offsets.
#include <cuda_runtime.h>

#include <algorithm>

#include "dd_internal.h"

namespace dd {

namespace {

constexpr int kAdjWarpChan = 8;                 // channels per warp
constexpr int kAdjWarps = 8;
constexpr int kAdjChan = kAdjWarpChan * kAdjWarps;  // channels per CTA
static_assert(kAdjChan == kAdjChanBlock, "adjoint span is planned for this block");
constexpr int kAdjSampPerThread = 8;
constexpr int kAdjTile = 32 * kAdjSampPerThread;  // raw samples per CTA
constexpr int kAdjDmChunk = 32;  // DMs staged per step (fewer when the windows are wide)

struct AdjRange {
  const int32_t* shifts;  // [n_dm][n_chan]
  const float* ybar;      // this range's plane [n_dm][n_out]
  int32_t n_dm;
  int32_t bin;
  int64_t n_out;
  int32_t win;            // staged window length per DM
};

struct AdjParams {
  AdjRange r[DD_MAX_RANGES];
  int32_t n_ranges;
  int32_t n_chan;
  int64_t n_samp;
  int64_t stride;
  int32_t max_win;
  int32_t dm_chunk;       // DMs staged per step (<= kAdjDmChunk)
};

__global__ void __launch_bounds__(256) adjoint_kernel(const AdjParams prm, float* __restrict__ xbar) {
  extern __shared__ unsigned char smem_raw[];
  float* win_buf = reinterpret_cast<float*>(smem_raw);                      // [chunk][max_win]
  int32_t* sh_buf = reinterpret_cast<int32_t*>(win_buf + prm.dm_chunk * prm.max_win);  // [chunk][64]
  int32_t* hi_buf = sh_buf + prm.dm_chunk * kAdjChan;                        // [chunk]

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int32_t n_cblk = (prm.n_chan + kAdjChan - 1) / kAdjChan;
  const int64_t tile = blockIdx.x / n_cblk;
  const int32_t c_first = (blockIdx.x % n_cblk) * kAdjChan;
  const int64_t t_raw0 = tile * kAdjTile;

  float acc[kAdjWarpChan][kAdjSampPerThread];
#pragma unroll
  for (int j = 0; j < kAdjWarpChan; ++j)
#pragma unroll
    for (int k = 0; k < kAdjSampPerThread; ++k) acc[j][k] = 0.f;

  for (int32_t ri = 0; ri < prm.n_ranges; ++ri) {
    const AdjRange rr = prm.r[ri];
    const int64_t u0 = t_raw0 / rr.bin;  // first decimated sample of the tile
    int32_t rel[kAdjSampPerThread];      // decimated offset of each of my samples
#pragma unroll
    for (int k = 0; k < kAdjSampPerThread; ++k)
      rel[k] = static_cast<int32_t>((t_raw0 + tx + 32 * k) / rr.bin - u0);

    for (int32_t d0 = 0; d0 < rr.n_dm; d0 += prm.dm_chunk) {
      const int32_t nd = min(prm.dm_chunk, rr.n_dm - d0);
      __syncthreads();
      // Shifts of the chunk's DMs for the CTA's channels (channels past the
      // last take its shifts; they are never written).
      for (int32_t e = tid; e < nd * kAdjChan; e += kAdjWarps * 32) {
        const int32_t dd = e / kAdjChan, cc = e % kAdjChan;
        const int32_t c = min(c_first + cc, prm.n_chan - 1);
        sh_buf[e] = rr.shifts[static_cast<int64_t>(d0 + dd) * prm.n_chan + c];
      }
      __syncthreads();
      // Warp ty stages DMs ty, ty + 8, ...: the row window from the block's
      // largest shift, ybar[d][u0 - hi + k], k < win (0 outside [0, n_out)).
      for (int32_t dd = ty; dd < nd; dd += kAdjWarps) {
        const int32_t hi = __reduce_max_sync(
            0xffffffffu, max(sh_buf[dd * kAdjChan + tx], sh_buf[dd * kAdjChan + 32 + tx]));
        if (tx == 0) hi_buf[dd] = hi;
        const float* yrow = rr.ybar + static_cast<int64_t>(d0 + dd) * rr.n_out;
        for (int32_t k = tx; k < rr.win; k += 32) {
          const int64_t u = u0 - hi + k;
          win_buf[dd * prm.max_win + k] = (u >= 0 && u < rr.n_out) ? yrow[u] : 0.f;
        }
      }
      __syncthreads();
      for (int32_t dd = 0; dd < nd; ++dd) {
        const int32_t hi = hi_buf[dd];
        const float* w = win_buf + dd * prm.max_win + hi;
        const int32_t* sh = sh_buf + dd * kAdjChan + ty * kAdjWarpChan;
#pragma unroll
        for (int j = 0; j < kAdjWarpChan; ++j) {
          const float* wj = w - sh[j];
#pragma unroll
          for (int k = 0; k < kAdjSampPerThread; ++k) acc[j][k] += wj[rel[k]];
        }
      }
    }
  }

#pragma unroll
  for (int j = 0; j < kAdjWarpChan; ++j) {
    const int32_t c = c_first + ty * kAdjWarpChan + j;
    if (c >= prm.n_chan) continue;
    float* xrow = xbar + static_cast<int64_t>(c) * prm.stride;
#pragma unroll
    for (int k = 0; k < kAdjSampPerThread; ++k) {
      const int64_t t = t_raw0 + tx + 32 * k;
      if (t < prm.n_samp) xrow[t] = acc[j][k];
    }
  }
}

// xbar[c][t] = sum_r z_r[n_chan - 1 - c][floor(t / b_r)]: the per-range
// adjoints computed by the forward pattern kernel (rows in reverse channel
// order, one sample per decimated sample) expanded over their time bins.
struct ExpandRange {
  const float* z;  // [n_chan][u_len]
  int64_t u_len;
  int32_t bin;
};
struct ExpandParams {
  ExpandRange r[DD_MAX_RANGES];
  int32_t n_ranges;
  int32_t n_chan;
  int64_t n_samp;
  int64_t stride;
};

__global__ void __launch_bounds__(256) adjoint_expand_kernel(const ExpandParams prm,
                                                             float* __restrict__ xbar) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x;
  const int32_t c = blockIdx.y;
  if (t >= prm.n_samp) return;
  float v = 0.f;
  for (int32_t i = 0; i < prm.n_ranges; ++i) {
    const ExpandRange& r = prm.r[i];
    v += r.z[static_cast<int64_t>(prm.n_chan - 1 - c) * r.u_len + t / r.bin];
  }
  xbar[static_cast<int64_t>(c) * prm.stride + t] = v;
}

// The padded cotangent rows of one range as the float-pair words the kF32P
// pattern tile reads: word u of row d is (Z[d][u], Z[d][u + pair]) with
// Z[d][u] = ybar[d][u - pad] for 0 <= u - pad < n_out and 0 elsewhere (the
// rows padded with pad = s_max zeros on both sides), u < stride.  Each thread
// writes 4 words.
__global__ void __launch_bounds__(256) adjoint_pack_kernel(const float* __restrict__ ybar,
                                                           int64_t n_out, int32_t pad,
                                                           int32_t pair, int64_t stride,
                                                           int64_t chunks_per_row, int64_t n_dm,
                                                           float2* __restrict__ w) {
  const int64_t gid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t d = gid / chunks_per_row;
  const int64_t u = (gid - d * chunks_per_row) * 4;
  if (d >= n_dm || u >= stride) return;
  const float* row = ybar + d * n_out;
  auto z = [&](int64_t v) { return v >= pad && v - pad < n_out ? row[v - pad] : 0.f; };
  float4* dst = reinterpret_cast<float4*>(w + d * stride + u);
  dst[0] = make_float4(z(u), z(u + pair), z(u + 1), z(u + 1 + pair));
  dst[1] = make_float4(z(u + 2), z(u + 2 + pair), z(u + 3), z(u + 3 + pair));
}

constexpr int kAdjNotServed = -1;

// Per-range sizes of the pattern adjoint: decimated samples per row u_len,
// padded cotangent row stride (in the tile's staged elements: floats, or
// float-pair words), result row stride; scratch in floats.  A plan of one
// range at bin 1 writes its result straight into xbar (no result buffer).
struct AdjSizes {
  int64_t u_len[DD_MAX_RANGES], pad_stride[DD_MAX_RANGES], z_stride[DD_MAX_RANGES];
  size_t in_floats = 0, out_floats = 0;
  bool direct_out = false;
};

// Sizes, or false when some range has no pattern tables.
bool adjoint_sizes(const dd_plan_s* p, int64_t n_samp, AdjSizes* z) {
  const size_t n_r = p->ranges.size();
  if (p->adj.size() != n_r || n_r == 0 || p->n_chan > 65535 || n_samp <= 0) return false;
  for (const RangePlan& ar : p->adj)
    if (!ar.tile_ok) return false;
  z->direct_out = n_r == 1 && p->ranges[0].r.bin == 1;
  for (size_t i = 0; i < n_r; ++i) {
    const RangePlan& rp = p->ranges[i];
    const size_t per = tk::float_pairs(p->adj[i].tile_kind) ? 2 : 1;  // floats per element
    z->u_len[i] = (n_samp - 1) / rp.r.bin + 1;
    z->pad_stride[i] = (z->u_len[i] + rp.s_max + 3) / 4 * 4;
    z->z_stride[i] = (z->u_len[i] + 3) / 4 * 4;
    z->in_floats = std::max(z->in_floats, per * static_cast<size_t>(rp.n_dm) * z->pad_stride[i]);
    if (!z->direct_out) z->out_floats += static_cast<size_t>(p->n_chan) * z->z_stride[i];
  }
  return true;
}

// The adjoint through the forward pattern kernel (plan.cpp, build_adjoint_range):
// per range, the cotangent rows padded with s_max zeros on both sides (in the
// caller's scratch), the forward transform of them with the transposed shift
// table, then the expansion.  kAdjNotServed when some range has no such tables
// or the scratch is too small.
int launch_adjoint_pattern(const dd_plan_s* p, const float* d_ybar, float* d_xbar,
                           int64_t n_samp, int64_t stride, const int64_t* n_out,
                           const int64_t* out_off, void* d_scratch, size_t scratch_bytes,
                           void* stream) {
  AdjSizes zs;
  if (!d_scratch || !adjoint_sizes(p, n_samp, &zs) ||
      scratch_bytes < (zs.in_floats + zs.out_floats) * sizeof(float))
    return kAdjNotServed;
  const size_t n_r = p->ranges.size();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* x_pad = static_cast<float*>(d_scratch);
  float* z = x_pad + zs.in_floats;
  ExpandParams ep{};
  ep.n_ranges = static_cast<int32_t>(n_r);
  ep.n_chan = p->n_chan;
  ep.n_samp = n_samp;
  ep.stride = stride;
  const unsigned char* ws = static_cast<const unsigned char*>(p->d_ws);
  int32_t* err = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(p->d_ws) + tk::kStatusOffset);
  for (size_t i = 0; i < n_r; ++i) {
    const RangePlan& rp = p->ranges[i];
    const RangePlan& ar = p->adj[i];
    const int64_t pad = rp.s_max;
    if (tk::float_pairs(ar.tile_kind)) {
      // Padding and pair packing in one pass.
      const int64_t chunks = zs.pad_stride[i] / 4;
      const int64_t blocks = (chunks * rp.n_dm + 255) / 256;
      if (blocks > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
      adjoint_pack_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
          d_ybar + out_off[i], n_out[i], static_cast<int32_t>(pad), pack_pair(ar),
          zs.pad_stride[i], chunks, rp.n_dm, reinterpret_cast<float2*>(x_pad));
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return static_cast<int>(e);
    } else {
      cudaError_t e = cudaMemsetAsync(
          x_pad, 0, static_cast<size_t>(rp.n_dm) * zs.pad_stride[i] * sizeof(float), st);
      if (e == cudaSuccess && n_out[i] > 0)
        e = cudaMemcpy2DAsync(x_pad + pad, zs.pad_stride[i] * sizeof(float), d_ybar + out_off[i],
                              n_out[i] * sizeof(float), n_out[i] * sizeof(float),
                              static_cast<size_t>(rp.n_dm), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return static_cast<int>(e);
    }
    if (zs.direct_out && ar.tile_pattern) {
      // One range at bin 1: result row c' is xbar's row n_chan - 1 - c'.
      const int rc = launch_forward_pattern(p, ar, ws + ar.off_tile_recs, err, x_pad,
                                            zs.pad_stride[i], zs.u_len[i],
                                            d_xbar + static_cast<int64_t>(p->n_chan - 1) * stride,
                                            0, zs.u_len[i], stream, -stride);
      return rc;
    }
    const int rc = launch_forward_tiled_with_tables(p, ar, ws + ar.off_tile_recs, err, x_pad,
                                                    zs.pad_stride[i], zs.z_stride[i], z, 0,
                                                    zs.u_len[i], stream);
    if (rc != 0) return rc;
    ep.r[i] = ExpandRange{z, zs.z_stride[i], rp.r.bin};
    z += static_cast<size_t>(p->n_chan) * zs.z_stride[i];
  }
  const dim3 grid(static_cast<unsigned>((n_samp + 255) / 256), static_cast<unsigned>(p->n_chan));
  adjoint_expand_kernel<<<grid, 256, 0, st>>>(ep, d_xbar);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace

size_t adjoint_scratch_bytes(const dd_plan_s* p, int64_t n_samp) {
  AdjSizes zs;
  return adjoint_sizes(p, n_samp, &zs) ? (zs.in_floats + zs.out_floats) * sizeof(float) : 0;
}

int launch_adjoint(const dd_plan_s* p, const float* d_ybar, float* d_xbar, int64_t n_samp,
                   int64_t stride, const int64_t* n_out, const int64_t* out_off,
                   void* d_scratch, size_t scratch_bytes, void* stream) {
  const int fast = launch_adjoint_pattern(p, d_ybar, d_xbar, n_samp, stride, n_out, out_off,
                                          d_scratch, scratch_bytes, stream);
  if (fast != kAdjNotServed) return fast;
  AdjParams prm{};
  prm.n_ranges = static_cast<int32_t>(p->ranges.size());
  prm.n_chan = p->n_chan;
  prm.n_samp = n_samp;
  prm.stride = stride;
  int32_t max_win = 1;
  for (int32_t i = 0; i < prm.n_ranges; ++i) {
    const RangePlan& rp = p->ranges[i];
    AdjRange& a = prm.r[i];
    a.shifts = reinterpret_cast<const int32_t*>(static_cast<const unsigned char*>(p->d_ws) +
                                                rp.off_shifts);
    a.ybar = d_ybar + out_off[i];
    a.n_dm = static_cast<int32_t>(rp.n_dm);
    a.bin = rp.r.bin;
    a.n_out = n_out[i];
    // Decimated samples touched by one tile, plus the channel-block span.
    a.win = kAdjTile / rp.r.bin + 2 + rp.adj_span;
    max_win = std::max(max_win, a.win);
  }
  prm.max_win = max_win;
  const size_t per_dm = static_cast<size_t>(max_win) * sizeof(float) + (kAdjChan + 1) * sizeof(int32_t);
  const size_t smem_max = 200 * 1024;
  prm.dm_chunk = static_cast<int32_t>(std::min<size_t>(kAdjDmChunk, smem_max / per_dm));
  if (prm.dm_chunk < 1) return static_cast<int>(cudaErrorInvalidConfiguration);
  const size_t smem = static_cast<size_t>(prm.dm_chunk) * per_dm;
  cudaError_t e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  const int32_t n_cblk = (p->n_chan + kAdjChan - 1) / kAdjChan;
  const int64_t tiles = (n_samp + kAdjTile - 1) / kAdjTile;
  const int64_t grid = tiles * n_cblk;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  adjoint_kernel<<<static_cast<unsigned>(grid), dim3(32, kAdjWarps), smem,
                   static_cast<cudaStream_t>(stream)>>>(prm, d_xbar);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace dd
