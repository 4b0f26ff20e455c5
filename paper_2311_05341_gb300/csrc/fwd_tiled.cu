// fwd_tiled.cu -- register-tiled forward dedispersion kernels for sm_103a
// (uint8, uint16 and float32 input at time bin 1), standalone and persistent.
//
// Computes Eq. 3 (Algorithm 1): Y[d][t] = sum_c X[c][t + s(c, d)], with the
// output partition of the paper's GPU kernel (Sec. 4: a CTA owns D_dm x D_t
// outputs and threads keep accumulators in registers, Algorithm 3), organised
// for GB300's issue rate:
//
//  * CTA = W warps x 32 lanes owning dr * W consecutive DMs and one time tile.
//    Warp w owns DMs d0 + dr*w .. d0 + dr*w + dr - 1; every lane owns the same
//    dr DMs x 20 window words (uint8: 40 samples, two per word in 16-bit lanes
//    as in Sec. 4.1's SIMD-within-a-word, pairing samples u and u + 640;
//    uint16 / float32: 20 samples).
//  * Staging (Algorithm 3's B_loc): per channel, the raw bytes of the window
//    starting at t0 + s(c, d0) are fetched with one TMA bulk copy
//    (cp.async.bulk, 16-byte aligned, completion on an mbarrier), two stages
//    in flight; all threads then unpack them into 32-bit window words.
//  * Register reuse across DMs: each lane loads its 36-word window of a
//    channel once (9 x 16-byte shared loads, conflict-free with a 20-word lane
//    stride) and adds it into all dr DMs.  DM i's offset inside the window is
//    a per-(channel, warp) 4-bit value (the paper's T_diff * Delta t_pc of
//    Eq. 6, resolved to an integer on the host); a warp-uniform indexed branch
//    per DM selects the register slice (generated by gen_dispatch.py).
//  * Time binning (Sec. 5.3) is fused into the unpacking: at bin b a window
//    word is the sum of b consecutive raw samples (uint8 then uses one
//    decimated sample per word).
//  * Accumulators are widened (uint8 pairs: every 256 channels) or stored
//    through a transposed shared tile into the output rows with coalesced
//    accesses.
//
// The persistent batch kernel runs the same tile body over a work list of
// (job, DM block, time tile) items taken from a device counter.  Every wait
// on an mbarrier is bounded; on timeout the kernel records kErrTimeout in the
// status word and returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dd_internal.h"
#include "fwd_tiled.h"
#include "fwd_tiled_dispatch.inc"
#include "tile_common.cuh"

namespace dd {
namespace tk {

namespace {

struct Smem {
  uint32_t bar_base;  // 2 mbarriers
  Rec* recs;          // [2][NC]
  uint8_t* raw;       // [2][NC][lraw]
  uint32_t* pw;       // [NC][lp] window words
};

template <int NC>
__device__ __forceinline__ Smem smem_layout(unsigned char* smem, int32_t lraw) {
  constexpr size_t kRawOff = raw_offset(NC);
  Smem sm;
  sm.bar_base = smem_u32(smem);
  sm.recs = reinterpret_cast<Rec*>(smem + kRecOffset);
  sm.raw = smem + kRawOff;
  sm.pw = reinterpret_cast<uint32_t*>(sm.raw + 2 * NC * static_cast<size_t>(lraw));
  return sm;
}

template <int KIND, int DR>
__device__ __forceinline__ void dispatch(AccT<KIND> (&acc)[DR][kH], const AccT<KIND> (&R)[kWin],
                                         uint32_t dl) {
  uint32_t ix[DR];
#pragma unroll
  for (int i = 0; i < DR; ++i) ix[i] = (dl >> (4 * i)) & 15u;
  if constexpr (KIND == kF32) {
    if constexpr (DR == 1) DD_TILE_CHANNEL_F32_1(acc, R, ix);
    else if constexpr (DR == 2) DD_TILE_CHANNEL_F32_2(acc, R, ix);
    else if constexpr (DR == 4) DD_TILE_CHANNEL_F32_4(acc, R, ix);
    else if constexpr (DR == 6) DD_TILE_CHANNEL_F32_6(acc, R, ix);
    else DD_TILE_CHANNEL_F32_8(acc, R, ix);
  } else {
    if constexpr (DR == 1) DD_TILE_CHANNEL_U32_1(acc, R, ix);
    else if constexpr (DR == 2) DD_TILE_CHANNEL_U32_2(acc, R, ix);
    else if constexpr (DR == 4) DD_TILE_CHANNEL_U32_4(acc, R, ix);
    else if constexpr (DR == 6) DD_TILE_CHANNEL_U32_6(acc, R, ix);
    else DD_TILE_CHANNEL_U32_8(acc, R, ix);
  }
}

// One (DM block, time tile) work unit.  gstage counts pipeline stages across
// the work units a CTA runs, so mbarrier phases continue from unit to unit.
// Returns false after a bounded wait gave up (the status word is set).
template <int KIND, int DR, int NW, int NC>
__device__ __forceinline__ bool tile_body(const TileParams& p, const Smem& sm, int blk,
                                          int64_t tile, uint32_t& gstage) {
  constexpr int kThreads = NW * 32;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int64_t t0 = tile * tile_samples(KIND);
  const int n_st = (p.n_chan + NC - 1) / NC;

  const Rec* my_recs = static_cast<const Rec*>(p.recs) + static_cast<int64_t>(blk) * p.n_chan;
  auto base_of = [&](int st) -> int32_t {
    const int c = st * NC + tid;
    return (tid < NC && st < n_st && c < p.n_chan) ? my_recs[c].base : 0;
  };
  const ChannelRecs<NC, Rec> cr{my_recs, sm.recs, p.n_chan};
  auto issue = [&](int st, int buf, int32_t base) {
    issue_stage<KIND, NC>(p, sm.bar_base, sm.raw, st, buf, t0, base, tid, cr.src(st),
                          cr.bytes(st), cr.dst(buf));
  };
  if (tid <= NC) {
    // Shared memory read by an earlier unit of a persistent CTA is rewritten
    // by the copies: order those generic-proxy reads before them.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(0, gstage & 1, base_of(0));
    if (n_st > 1) issue(1, (gstage + 1) & 1, base_of(1));
  }
  int32_t next_base = base_of(2);

  AccT<KIND> acc[DR][kH];
#pragma unroll
  for (int i = 0; i < DR; ++i)
#pragma unroll
    for (int j = 0; j < kH; ++j) acc[i][j] = AccT<KIND>(0);

  bool first = true;
  int since = 0;  // channels accumulated since the last widen
  const int units = p.lp >> 2;

  for (int st = 0; st < n_st; ++st) {
    const uint32_t g = gstage + st;
    const int buf = g & 1;
    const uint32_t parity = (g >> 1) & 1;
    const bool ok = mbar_wait(sm.bar_base + 8u * buf, parity, p.wait_iters);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(p.err, kErrTimeout);
        // Let copies still in flight land before the CTA exits (bounded).
        if (st != p.hold_stage) mbar_wait(sm.bar_base + 8u * buf, parity);
        if (st + 1 < n_st && st + 1 != p.hold_stage)
          mbar_wait(sm.bar_base + 8u * (buf ^ 1), ((g + 1) >> 1) & 1);
      }
      return false;
    }
    const int nc = min(NC, p.n_chan - st * NC);

    {  // Unpack raw bytes into window words.
      const uint8_t* rawb = sm.raw + static_cast<size_t>(buf) * NC * p.lraw;
      const int total = nc * units;
      for (int u = tid; u < total; u += kThreads) {
        const int ch =
            static_cast<int>((static_cast<uint64_t>(u) * p.units_magic) >> (32 + p.units_shift));
        const int q = u - ch * units;
        const uint4 v = unpack_unit<KIND, kPair>(rawb + static_cast<size_t>(ch) * p.lraw, q, p.bin);
        *reinterpret_cast<uint4*>(sm.pw + static_cast<size_t>(ch) * p.lp + 4 * q) = v;
      }
    }
    __syncthreads();

    // Shift-and-sum.  The loop stays rolled so the dispatch block, and its PTX
    // labels, appear once per instantiation.
    const Rec* rs = sm.recs + buf * NC;
#pragma unroll 1
    for (int ch = 0; ch < nc; ++ch) {
      const uint32_t dl = rs[ch].delta[w];
      const int a = 4 * static_cast<int>(rs[ch].aq[w]);
      const uint4* src = reinterpret_cast<const uint4*>(sm.pw + static_cast<size_t>(ch) * p.lp +
                                                         kH * l + a);
      AccT<KIND> R[kWin];
#pragma unroll
      for (int k = 0; k < kWin / 4; ++k) {
        const uint4 v = src[k];
        if constexpr (KIND == kF32) {
          R[4 * k] = __uint_as_float(v.x);
          R[4 * k + 1] = __uint_as_float(v.y);
          R[4 * k + 2] = __uint_as_float(v.z);
          R[4 * k + 3] = __uint_as_float(v.w);
        } else {
          R[4 * k] = v.x;
          R[4 * k + 1] = v.y;
          R[4 * k + 2] = v.z;
          R[4 * k + 3] = v.w;
        }
      }
      dispatch<KIND, DR>(acc, R, dl);
    }
    since += nc;
    __syncthreads();  // window words, raw[buf] and recs[buf] are free

    if (tid <= NC && st + 2 < n_st) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(st + 2, buf, next_base);
      next_base = base_of(st + 3);
    }
    if (since + NC > p.flush || st == n_st - 1) {
      widen_store<KIND, DR, NW, NC, kH>(p, sm.pw, acc, blk, t0, first);
      first = false;
      since = 0;
    }
  }
  gstage += n_st;
  __syncthreads();  // the transpose tile (window buffer) is free for the next unit
  return true;
}

template <int NC>
__device__ __forceinline__ void init_barriers(const Smem& sm) {
  if (threadIdx.x == 0) {
    mbar_init(sm.bar_base, NC + 1);
    mbar_init(sm.bar_base + 8, NC + 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

}  // namespace

template <int KIND, int DR, int NW, int MINB, int NC>
__global__ void __launch_bounds__(NW * 32, MINB) fwd_tiled_kernel(const TileParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Smem sm = smem_layout<NC>(smem, p.lraw);
  init_barriers<NC>(sm);
  uint32_t gstage = 0;
  tile_body<KIND, DR, NW, NC>(p, sm, blockIdx.x % p.n_blocks, blockIdx.x / p.n_blocks + p.tile0,
                              gstage);
}

// One batch item of one variant.  Returns the continued stage count, or
// kStageError after a timeout.
constexpr uint32_t kStageError = 0xffffffffu;

template <int KIND, int DR, int NW, int NC>
__device__ __forceinline__ uint32_t batch_item(const BatchJob* job, int blk, int tile,
                                            uint32_t gstage, unsigned char* smem,
                                            int32_t max_lraw) {
  const Smem sm = smem_layout<NC>(smem, max_lraw);
  // Parameters read from global memory as needed (read-only for the launch).
  const TileParams& p = static_cast<const BatchJob* __restrict__>(job)->p;
  uint32_t g = gstage;
  return tile_body<KIND, DR, NW, NC>(p, sm, blk, tile, g) ? g : kStageError;
}

template <int NW, int MINB, int NC>
__global__ void __launch_bounds__(NW * 32, MINB) fwd_batch_kernel(const BatchArgs b) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int item_slot;
  init_barriers<NC>(smem_layout<NC>(smem, b.max_lraw));
  uint32_t g = 0;
  for (;;) {
    if (threadIdx.x == 0) item_slot = static_cast<int>(atomicAdd(b.counter, 1u));
    __syncthreads();
    const int it = item_slot;
    if (it >= b.n_items) break;
    const BatchItem item = b.items[it];
    const BatchJob* job = b.jobs + item.job;
    // The shared-memory layout is sized for the largest raw window and window
    // of any job; a job indexes the raw buffers with its own (smaller) lraw.
    switch (job->kind * 16 + job->dr) {
      case kU8 * 16 + 4: g = batch_item<kU8, 4, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kU8 * 16 + 2: g = batch_item<kU8, 2, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kU8 * 16 + 1: g = batch_item<kU8, 1, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kU8W * 16 + 4: g = batch_item<kU8W, 4, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kU8W * 16 + 2: g = batch_item<kU8W, 2, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kU8W * 16 + 1: g = batch_item<kU8W, 1, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kU16 * 16 + 4: g = batch_item<kU16, 4, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kU16 * 16 + 2: g = batch_item<kU16, 2, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kU16 * 16 + 1: g = batch_item<kU16, 1, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kF32 * 16 + 4: g = batch_item<kF32, 4, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kF32 * 16 + 2: g = batch_item<kF32, 2, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      case kF32 * 16 + 1: g = batch_item<kF32, 1, NW, NC>(job, item.blk, item.tile, g, smem, b.max_lraw); break;
      default: break;
    }
    if (g == kStageError) break;
  }
}

}  // namespace tk

namespace {

template <int KIND, int DR, int NW, int MINB, int NC>
int launch_tiled_shape(const tk::TileParams& prm, int64_t grid, cudaStream_t st) {
  const tk::Shape* sh = tk::shape_for(DR);
  const size_t smem = tk::smem_bytes(KIND, prm.bin, *sh, prm.lp);
  auto kern = tk::fwd_tiled_kernel<KIND, DR, NW, MINB, NC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  kern<<<static_cast<unsigned>(grid), NW * 32, smem, st>>>(prm);
  return static_cast<int>(cudaGetLastError());
}

template <int KIND>
int launch_kind(int dr, const tk::TileParams& prm, int64_t grid, cudaStream_t st) {
  switch (dr) {
    case 8: return launch_tiled_shape<KIND, 8, 8, 1, 16>(prm, grid, st);
    case 6: return launch_tiled_shape<KIND, 6, 12, 1, 24>(prm, grid, st);
    case 4: return launch_tiled_shape<KIND, 4, 12, 1, 24>(prm, grid, st);
    case 2: return launch_tiled_shape<KIND, 2, 12, 1, 16>(prm, grid, st);
    case 1: return launch_tiled_shape<KIND, 1, 12, 1, 16>(prm, grid, st);
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

}  // namespace

tk::TileParams tiled_params(const dd_plan_s* p, const RangePlan& rp, const void* recs,
                            int32_t* err, const void* d_in, int64_t stride, int64_t n_out,
                            void* d_out, int kind, bool widen_slots) {
  // The tables were built for rp.tile_kind; `kind` (a packed-copy kind, see
  // copy_kind) may run them from a packed copy of the input.
  if (kind <= 0) kind = rp.tile_kind;
  tk::TileParams prm{};
  prm.x = d_in;
  prm.stride = stride;
  prm.x_origin = 0;
  prm.align = tk::align_samples(rp.tile_kind, tk::staged_bin(rp.tile_kind, rp.r.bin));
  prm.n_chan = rp.tile_n_chan > 0 ? rp.tile_n_chan : p->n_chan;
  prm.recs = recs;
  if (rp.tile_pattern && rp.tile_chunk_bytes > 0) {  // pair tiles: base table, then chunks
    prm.bases = static_cast<const int32_t*>(recs);
    prm.recs = static_cast<const unsigned char*>(recs) + rp.tile_chunk_off;
    prm.chunk_bytes = rp.tile_chunk_bytes;
  }
  prm.n_dm = static_cast<int32_t>(rp.n_dm);
  prm.n_blocks = rp.tile_n_blocks;
  prm.n_out = n_out;
  prm.out_stride = n_out;
  prm.tile0 = 0;
  prm.t_end = n_out;
  prm.lp = rp.tile_lp;
  const int sb = tk::staged_bin(kind, rp.r.bin);  // packed copies: already decimated
  prm.lraw = rp.tile_pattern
                 ? tk::pat_raw_bytes(kind, sb, tk::kPatShapes[rp.tile_shape], rp.tile_lp)
                 : tk::raw_bytes(kind, sb, rp.tile_lp);
  prm.units_magic = rp.tile_units_magic;
  prm.units_shift = rp.tile_units_shift;
  prm.bin = sb;
  prm.flush = tk::flush_channels(kind, rp.r.bin);
  // Packed 4-bit input: at most 15 per sample in the 16-bit lanes.
  if (kind == tk::kU8P && p->dtype == DD_U4) prm.flush = tk::flush_channels(tk::kU4, 1);
  prm.out = d_out;
  prm.err = err;
  prm.wait_iters = p->wait_iters;
  prm.hold_stage = p->hold_stage;
  // Pattern tiles with 16-bit lanes widen into the workspace's slots when the
  // plan has a bound workspace with them (the no-allocation entry point's
  // tables live elsewhere and widen into the output rows).
  prm.wslots = nullptr;
  prm.wflags = nullptr;
  prm.n_wslots = 0;
  prm.wslot_words = 0;
  const int32_t need = tk::kPatDr * (rp.tile_pattern ? tk::kPatShapes[rp.tile_shape].warps : 0) *
                       32 * rp.tile_h;
  if (widen_slots && rp.tile_pattern && tk::packed_pairs(kind) && p->d_ws &&
      p->wslot_words >= need) {
    unsigned char* ws = static_cast<unsigned char*>(p->d_ws);
    prm.wslots = reinterpret_cast<unsigned long long*>(ws + p->off_wslots);
    prm.wflags = reinterpret_cast<int32_t*>(ws + p->off_wflags);
    prm.n_wslots = tk::kWidenSlots;
    prm.wslot_words = p->wslot_words;
  }
  return prm;
}

int64_t range_tile_samples(const RangePlan& rp) {
  if (!rp.tile_ok) return kGenSampPerCta;
  return rp.tile_pattern ? tk::pat_tile_samples(rp.tile_kind, rp.tile_h)
                         : tk::tile_samples(rp.tile_kind);
}

int launch_forward_tiled_with_tables(const dd_plan_s* p, const RangePlan& rp, const void* recs,
                                     int32_t* err, const void* d_in, int64_t stride,
                                     int64_t n_out, void* d_out, int64_t t_begin, int64_t t_end,
                                     void* stream, bool widen_slots) {
  if (rp.tile_pattern)
    return launch_forward_pattern(p, rp, recs, err, d_in, stride, n_out, d_out, t_begin, t_end,
                                  stream, n_out, 0, 0, widen_slots);
  tk::TileParams prm = tiled_params(p, rp, recs, err, d_in, stride, n_out, d_out);
  const int ts = tk::tile_samples(rp.tile_kind);
  if (t_begin % ts != 0 || t_begin < 0 || t_end > n_out || t_end <= t_begin)
    return static_cast<int>(cudaErrorInvalidValue);
  prm.tile0 = t_begin / ts;
  prm.t_end = t_end;
  const int64_t tiles = (t_end + ts - 1) / ts - prm.tile0;
  const int64_t grid = tiles * rp.tile_n_blocks;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (rp.tile_kind) {
    case tk::kU8: return launch_kind<tk::kU8>(rp.tile_dr, prm, grid, st);
    case tk::kU8W: return launch_kind<tk::kU8W>(rp.tile_dr, prm, grid, st);
    case tk::kU16: return launch_kind<tk::kU16>(rp.tile_dr, prm, grid, st);
    case tk::kF32: return launch_kind<tk::kF32>(rp.tile_dr, prm, grid, st);
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

int launch_forward_tiled(const dd_plan_s* p, const RangePlan& rp, const void* d_in,
                         int64_t stride, int64_t n_samp, int64_t n_out, void* d_out,
                         int64_t t_begin, int64_t t_end, void* stream) {
  (void)n_samp;
  const unsigned char* ws = static_cast<const unsigned char*>(p->d_ws);
  return launch_forward_tiled_with_tables(
      p, rp, ws + rp.off_tile_recs,
      reinterpret_cast<int32_t*>(static_cast<unsigned char*>(p->d_ws) + tk::kStatusOffset), d_in,
      stride, n_out, d_out, t_begin, t_end, stream);
}

int launch_batch(const tk::BatchArgs& args, int32_t grid, size_t smem, void* stream) {
  auto kern = tk::fwd_batch_kernel<tk::kBatchWarps, 1, tk::kBatchNc>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  kern<<<grid, 12 * 32, smem, static_cast<cudaStream_t>(stream)>>>(args);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace dd
