// pattern_kernels.cuh -- the pattern-tile kernels (pattern_body.cuh) and their
// launch templates: the one-unit-per-CTA kernel of dd_run and the persistent
// kernel of dd_batch_run, for every tk::kPatShapes entry that serves a kind.
// Included only by the per-kind translation units fwd_pattern_k*.cu (one-unit
// kernels) and fwd_pattern_batch_k*.cu (persistent kernels), each of which
// defines one kind's launcher, so that they compile in parallel;
// fwd_pattern.cu and fwd_pattern_batch.cu dispatch on the kind.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <iterator>
#include <utility>

#include "dd_internal.h"
#include "pattern_body.cuh"

namespace dd {
namespace tk {

template <int KIND, int H, int NW, int NC, bool PAIRS, bool DBUF, int AMAX, int SLOTS>
__global__ void __launch_bounds__(NW * 32, 1) fwd_pattern_kernel(const TileParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  using namespace pattern;
  const PSmem sm = pat_layout<NW, NC, PAIRS, DBUF>(smem, p.lraw);
  if (threadIdx.x == 0) {
    mbar_init(sm.bar_base, NC + 1);
    mbar_init(sm.bar_base + 8, NC + 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int blk = blockIdx.x % p.n_blocks;
  const int64_t tile = blockIdx.x / p.n_blocks + p.tile0;
  pat_body<KIND, H, NW, NC, PAIRS, DBUF, AMAX, SLOTS>(p, sm, blk, tile);
}

}  // namespace tk

namespace pattern_launch {

template <int KIND, int H, int NW, int NC, bool PAIRS, bool DBUF, int AMAX, int SLOTS>
int launch_pattern_mode(const tk::TileParams& prm, int64_t grid, cudaStream_t st) {
  const size_t smem =
      tk::pat_smem_bytes(KIND, prm.bin, tk::PatShape{H, NW, NC, PAIRS, DBUF, AMAX}, prm.lp);
  auto kern = tk::fwd_pattern_kernel<KIND, H, NW, NC, PAIRS, DBUF, AMAX, SLOTS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  kern<<<static_cast<unsigned>(grid), NW * 32, smem, st>>>(prm);
  return static_cast<int>(cudaGetLastError());
}

template <int KIND, int H, int NW, int NC, bool PAIRS, bool DBUF, int AMAX>
int launch_pattern_shape(const tk::TileParams& prm, int64_t grid, cudaStream_t st) {
  if constexpr (tk::packed_pairs(KIND)) {
    switch (tk::widen_mode(KIND, NC, prm.wslots != nullptr, prm.flush)) {
      case 8: return launch_pattern_mode<KIND, H, NW, NC, PAIRS, DBUF, AMAX, 8>(prm, grid, st);
      case 1: return launch_pattern_mode<KIND, H, NW, NC, PAIRS, DBUF, AMAX, 1>(prm, grid, st);
      default: break;
    }
    if constexpr (KIND == tk::kU8P) {
      switch (tk::widen_mode(KIND, NC, prm.wslots != nullptr, prm.flush)) {
        case 4: return launch_pattern_mode<KIND, H, NW, NC, PAIRS, DBUF, AMAX, 4>(prm, grid, st);
        case 2: return launch_pattern_mode<KIND, H, NW, NC, PAIRS, DBUF, AMAX, 2>(prm, grid, st);
        default: break;
      }
    }
  }
  return launch_pattern_mode<KIND, H, NW, NC, PAIRS, DBUF, AMAX, 0>(prm, grid, st);
}

template <int KIND, int I>
int launch_pattern_index(const tk::TileParams& prm, int64_t grid, cudaStream_t st) {
  constexpr tk::PatShape s = tk::kPatShapes[I];
  if constexpr (!tk::pat_shape_serves(s, KIND)) {
    return static_cast<int>(cudaErrorInvalidValue);  // the planner never picks it
  } else {
    return launch_pattern_shape<KIND, s.h, s.warps, s.nc, s.pairs, s.dbuf, s.amax>(
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

}  // namespace pattern_launch

namespace tk {

__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Persistent kernel of one variant (KIND, kPatShapes[I]): the jobs of a batch
// are grouped by variant and each group is one launch, so every launch has
// the register allocation of its own variant.
template <int KIND, int I, int SLOTS>
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
        pattern::pat_layout<s.warps, s.nc, s.pairs, s.dbuf>(smem, p.lraw);
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
    const bool ok = pattern::pat_body<KIND, s.h, s.warps, s.nc, s.pairs, s.dbuf, s.amax, SLOTS>(
        p, sm, item.blk, item.tile);
    if (!ok) break;
  }
}

}  // namespace tk

namespace pattern_launch {

template <int KIND, int I, int SLOTS>
int launch_variant_mode(const tk::PatBatchArgs& args, int32_t grid, size_t smem,
                        cudaStream_t st) {
  auto kern = tk::fwd_pattern_batch_kernel<KIND, I, SLOTS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  kern<<<grid, tk::kPatShapes[I].warps * 32, smem, st>>>(args);
  return static_cast<int>(cudaGetLastError());
}

// mode: the widening mode every job of the launch takes (tk::widen_mode).
template <int KIND, int I>
int launch_variant(const tk::PatBatchArgs& args, int32_t grid, size_t smem, cudaStream_t st,
                   int mode) {
  if constexpr (!tk::pat_shape_serves(tk::kPatShapes[I], KIND)) {
    return static_cast<int>(cudaErrorInvalidValue);  // never grouped by the host
  } else {
    if constexpr (tk::packed_pairs(KIND)) {
      if (mode == 8) return launch_variant_mode<KIND, I, 8>(args, grid, smem, st);
      if (mode == 1) return launch_variant_mode<KIND, I, 1>(args, grid, smem, st);
    }
    if constexpr (KIND == tk::kU8P) {
      if (mode == 4) return launch_variant_mode<KIND, I, 4>(args, grid, smem, st);
      if (mode == 2) return launch_variant_mode<KIND, I, 2>(args, grid, smem, st);
    }
    return launch_variant_mode<KIND, I, 0>(args, grid, smem, st);
  }
}

template <int KIND, size_t... I>
int launch_kind(int shape, const tk::PatBatchArgs& args, int32_t grid, size_t smem,
                cudaStream_t st, int mode, std::index_sequence<I...>) {
  int rc = static_cast<int>(cudaErrorInvalidValue);
  ((shape == static_cast<int>(I)
        ? (rc = launch_variant<KIND, I>(args, grid, smem, st, mode), 0)
        : 0),
   ...);
  return rc;
}

}  // namespace pattern_launch

}  // namespace dd

// The launchers of one kind (declared in dd_internal.h): the one-unit kernel
// (DD_PATTERN_KIND_FORWARD) and the persistent batch kernel
// (DD_PATTERN_KIND_BATCH), each in a translation unit of its own.
#define DD_PATTERN_KIND_FORWARD(K)                                                          \
  namespace dd {                                                                            \
  int pattern_forward_##K(int shape, const tk::TileParams& prm, int64_t grid, void* st) {   \
    return pattern_launch::launch_pattern_kind<tk::K>(shape, prm, grid,                    \
                                                      static_cast<cudaStream_t>(st));       \
  }                                                                                         \
  }
#define DD_PATTERN_KIND_BATCH(K)                                                            \
  namespace dd {                                                                            \
  int pattern_batch_##K(int shape, const tk::PatBatchArgs& args, int32_t grid, size_t smem, \
                        void* st, int mode) {                                               \
    return pattern_launch::launch_kind<tk::K>(                                              \
        shape, args, grid, smem, static_cast<cudaStream_t>(st), mode,                       \
        std::make_index_sequence<tk::kNumPatShapes>{});                                     \
  }                                                                                         \
  }
