// fwd_pattern.cu -- the pattern tiles launched one (DM block, time tile)
// unit per CTA: the launch geometry, and the dispatch on the window-word kind
// to the per-kind launchers (fwd_pattern_k*.cu, pattern_kernels.cuh).
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace dd {

int launch_forward_pattern(const dd_plan_s* p, const RangePlan& rp, const void* recs,
                           int32_t* err, const void* d_in, int64_t stride, int64_t n_out,
                           void* d_out, int64_t t_begin, int64_t t_end, void* stream,
                           int64_t out_stride, int kind, int64_t x_origin, bool widen_slots) {
  if (kind <= 0) kind = rp.tile_kind;
  tk::TileParams prm =
      tiled_params(p, rp, recs, err, d_in, stride, n_out, d_out, kind, widen_slots);
  prm.out_stride = out_stride;
  prm.x_origin = x_origin;
  if (x_origin < 0 || x_origin % prm.align != 0) return static_cast<int>(cudaErrorInvalidValue);
  const int ts = tk::pat_tile_samples(kind, rp.tile_h);
  if (t_begin % ts != 0 || t_begin < 0 || t_end > n_out || t_end <= t_begin)
    return static_cast<int>(cudaErrorInvalidValue);
  prm.tile0 = t_begin / ts;
  prm.t_end = t_end;
  const int64_t tiles = (t_end + ts - 1) / ts - prm.tile0;
  const int64_t grid = tiles * rp.tile_n_blocks;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  const int shape = rp.tile_shape;
  switch (kind) {
#define DD_CASE(K) \
  case tk::K: return pattern_forward_##K(shape, prm, grid, stream);
    DD_PATTERN_KINDS(DD_CASE)
#undef DD_CASE
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

}  // namespace dd
