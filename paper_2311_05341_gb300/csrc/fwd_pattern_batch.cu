// fwd_pattern_batch.cu -- persistent batch kernels of the pattern tiles.
//
// One CTA per SM takes (job, DM block, time tile) items from a device counter
// until the list is exhausted; each item runs the pattern work unit
// (pattern_body.cuh).  One kernel per variant (kind, tk::kPatShapes entry):
// the host groups a batch's jobs by variant and launches each group.
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "dd_internal.h"
#include "pattern_body.cuh"

namespace dd {
namespace tk {

namespace {

__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

}  // namespace

// Persistent kernel of one variant (KIND, kPatShapes[I]): the jobs of a batch
// are grouped by variant and each group is one launch, so every launch has
// the register allocation of its own variant.
template <int KIND, int I>
__global__ void __launch_bounds__(kPatShapes[I].warps * 32, 1)
    fwd_pattern_batch_kernel(const PatBatchArgs b) {
  constexpr PatShape s = kPatShapes[I];
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int item_slot;
  bool barriers_valid = false;
  for (;;) {
    if (threadIdx.x == 0) item_slot = static_cast<int>(atomicAdd(b.counter, 1u));
    __syncthreads();
    const int it = item_slot;
    if (it >= b.n_items) break;
    const BatchItem item = b.items[it];
    // The job's parameters stay in global memory (read-only for the launch):
    // a copy in registers would crowd out the accumulators.
    const TileParams& p = static_cast<const PatBatchJob* __restrict__>(b.jobs)[item.job].p;
    const pattern::PSmem sm =
        pattern::pat_layout<s.warps, s.nc, s.pairs, s.dbuf, s.merge>(smem, p.lraw);
    __syncthreads();  // every thread has read item_slot; the previous item is done
    if (threadIdx.x == 0) {
      // Stage phases restart at 0 for every item: re-initialise the barriers
      // (all copies of the previous item have landed and been waited for).
      if (barriers_valid) {
        mbar_inval(sm.bar_base);
        mbar_inval(sm.bar_base + 8);
      }
      mbar_init(sm.bar_base, s.nc + 1);
      mbar_init(sm.bar_base + 8, s.nc + 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    barriers_valid = true;
    __syncthreads();
    bool ok;
    if constexpr (s.merge)
      ok = pattern::pat_body_merge<s.h, s.warps, s.nc, s.amax>(p, sm, item.blk, item.tile);
    else
      ok = pattern::pat_body<KIND, s.h, s.warps, s.nc, s.pairs, s.dbuf, s.amax>(p, sm, item.blk,
                                                                               item.tile);
    if (!ok) break;
  }
}

}  // namespace tk

namespace {

template <int KIND, int I>
int launch_variant(const tk::PatBatchArgs& args, int32_t grid, size_t smem, cudaStream_t st) {
  if constexpr (!tk::pat_shape_serves(tk::kPatShapes[I], KIND)) {
    return static_cast<int>(cudaErrorInvalidValue);  // never grouped by the host
  } else {
    auto kern = tk::fwd_pattern_batch_kernel<KIND, I>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return static_cast<int>(e);
    kern<<<grid, tk::kPatShapes[I].warps * 32, smem, st>>>(args);
    return static_cast<int>(cudaGetLastError());
  }
}

template <int KIND, size_t... I>
int launch_kind(int shape, const tk::PatBatchArgs& args, int32_t grid, size_t smem,
                cudaStream_t st, std::index_sequence<I...>) {
  int rc = static_cast<int>(cudaErrorInvalidValue);
  ((shape == static_cast<int>(I) ? (rc = launch_variant<KIND, I>(args, grid, smem, st), 0) : 0),
   ...);
  return rc;
}

}  // namespace

int launch_pattern_batch(int kind, int shape, const tk::PatBatchArgs& args, int32_t grid,
                         size_t smem, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  constexpr auto kShapes = std::make_index_sequence<tk::kNumPatShapes>{};
  switch (kind) {
    case tk::kU8: return launch_kind<tk::kU8>(shape, args, grid, smem, st, kShapes);
    case tk::kU8W: return launch_kind<tk::kU8W>(shape, args, grid, smem, st, kShapes);
    case tk::kU16: return launch_kind<tk::kU16>(shape, args, grid, smem, st, kShapes);
    case tk::kU4: return launch_kind<tk::kU4>(shape, args, grid, smem, st, kShapes);
    case tk::kF32: return launch_kind<tk::kF32>(shape, args, grid, smem, st, kShapes);
    case tk::kF32D: return launch_kind<tk::kF32D>(shape, args, grid, smem, st, kShapes);
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

}  // namespace dd
