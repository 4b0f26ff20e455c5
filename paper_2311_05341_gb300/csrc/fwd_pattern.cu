// fwd_pattern.cu -- the pattern tiles (pattern_body.cuh) launched one
// (DM block, time tile) unit per CTA, for every kind and shape of
// tk::kPatShapes that serves it.
#include <cuda_runtime.h>

#include <cstdint>
#include <iterator>
#include <utility>

#include "dd_internal.h"
#include "pattern_body.cuh"

namespace dd {
namespace tk {

template <int KIND, int H, int NW, int NC, bool PAIRS, bool DBUF, int AMAX, bool MERGE>
__global__ void __launch_bounds__(NW * 32, 1) fwd_pattern_kernel(const TileParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  using namespace pattern;
  const PSmem sm = pat_layout<NW, NC, PAIRS, DBUF, MERGE>(smem, p.lraw);
  if (threadIdx.x == 0) {
    mbar_init(sm.bar_base, NC + 1);
    mbar_init(sm.bar_base + 8, NC + 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int blk = blockIdx.x % p.n_blocks;
  const int64_t tile = blockIdx.x / p.n_blocks + p.tile0;
  if constexpr (MERGE) pat_body_merge<H, NW, NC, AMAX>(p, sm, blk, tile);
  else pat_body<KIND, H, NW, NC, PAIRS, DBUF, AMAX>(p, sm, blk, tile);
}

}  // namespace tk

namespace {

template <int KIND, int H, int NW, int NC, bool PAIRS, bool DBUF, int AMAX, bool MERGE>
int launch_pattern_shape(const tk::TileParams& prm, int64_t grid, cudaStream_t st) {
  const size_t smem = tk::pat_smem_bytes(
      KIND, prm.bin, tk::PatShape{H, NW, NC, PAIRS, DBUF, AMAX, MERGE}, prm.lp, prm.nv);
  auto kern = tk::fwd_pattern_kernel<KIND, H, NW, NC, PAIRS, DBUF, AMAX, MERGE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  kern<<<static_cast<unsigned>(grid), NW * 32, smem, st>>>(prm);
  return static_cast<int>(cudaGetLastError());
}

template <int KIND, int I>
int launch_pattern_index(const tk::TileParams& prm, int64_t grid, cudaStream_t st) {
  constexpr tk::PatShape s = tk::kPatShapes[I];
  if constexpr (!tk::pat_shape_serves(s, KIND)) {
    return static_cast<int>(cudaErrorInvalidValue);  // the planner never picks it
  } else {
    return launch_pattern_shape<KIND, s.h, s.warps, s.nc, s.pairs, s.dbuf, s.amax, s.merge>(
        prm, grid, st);
  }
}

template <int KIND, size_t... I>
int launch_pattern_kind(int shape, const tk::TileParams& prm, int64_t grid, cudaStream_t st,
                        std::index_sequence<I...>) {
  int rc = static_cast<int>(cudaErrorInvalidValue);
  ((shape == static_cast<int>(I) ? (rc = launch_pattern_index<KIND, I>(prm, grid, st), 0) : 0),
   ...);
  return rc;
}

template <int KIND>
int launch_pattern_kind(int shape, const tk::TileParams& prm, int64_t grid, cudaStream_t st) {
  return launch_pattern_kind<KIND>(
      shape, prm, grid, st, std::make_index_sequence<std::size(tk::kPatShapes)>{});
}

}  // namespace

int launch_forward_pattern(const dd_plan_s* p, const RangePlan& rp, const void* recs,
                           int32_t* err, const void* d_in, int64_t stride, int64_t n_out,
                           void* d_out, int64_t t_begin, int64_t t_end, void* stream) {
  tk::TileParams prm = tiled_params(p, rp, recs, err, d_in, stride, n_out, d_out);
  const int ts = tk::pat_tile_samples(rp.tile_kind, rp.tile_h);
  if (t_begin % ts != 0 || t_begin < 0 || t_end > n_out || t_end <= t_begin)
    return static_cast<int>(cudaErrorInvalidValue);
  prm.tile0 = t_begin / ts;
  prm.t_end = t_end;
  const int64_t tiles = (t_end + ts - 1) / ts - prm.tile0;
  const int64_t grid = tiles * rp.tile_n_blocks;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (rp.tile_kind) {
    case tk::kU8: return launch_pattern_kind<tk::kU8>(rp.tile_shape, prm, grid, st);
    case tk::kU8W: return launch_pattern_kind<tk::kU8W>(rp.tile_shape, prm, grid, st);
    case tk::kU16: return launch_pattern_kind<tk::kU16>(rp.tile_shape, prm, grid, st);
    case tk::kU4: return launch_pattern_kind<tk::kU4>(rp.tile_shape, prm, grid, st);
    case tk::kU8P: return launch_pattern_kind<tk::kU8P>(rp.tile_shape, prm, grid, st);
    case tk::kF32D: return launch_pattern_kind<tk::kF32D>(rp.tile_shape, prm, grid, st);
    case tk::kU16P: return launch_pattern_kind<tk::kU16P>(rp.tile_shape, prm, grid, st);
    case tk::kF32: return launch_pattern_kind<tk::kF32>(rp.tile_shape, prm, grid, st);
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

}  // namespace dd
