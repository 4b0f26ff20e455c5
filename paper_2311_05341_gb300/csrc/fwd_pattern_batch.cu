// fwd_pattern_batch.cu -- persistent batch kernels of the pattern tiles.
//
// One CTA per SM takes (job, DM block, time tile) items from a device counter
// until the list is exhausted; each item runs the pattern work unit
// (pattern_body.cuh).  One kernel per variant (kind, tk::kPatShapes entry):
// the host groups a batch's jobs by variant and launches each group.  The
// kernels live in pattern_kernels.cuh, instantiated per kind in
// fwd_pattern_k*.cu; this file dispatches on the kind.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace dd {

int launch_pattern_batch(int kind, int shape, const tk::PatBatchArgs& args, int32_t grid,
                         size_t smem, void* stream, int mode) {
  switch (kind) {
#define DD_CASE(K) \
  case tk::K: return pattern_batch_##K(shape, args, grid, smem, stream, mode);
    DD_PATTERN_KINDS(DD_CASE)
#undef DD_CASE
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

}  // namespace dd
