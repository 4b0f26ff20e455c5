// tile_common.cuh -- device helpers shared by the register-tiled forward
// kernels (fwd_tiled.cu, fwd_pattern.cu): TMA bulk copies completing on
// mbarriers, bounded mbarrier waits, accumulator/output types and the
// unpacking of staged raw bytes into 32-bit window words (time binning fused).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "fwd_tiled.h"

namespace dd {
namespace tk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Bounded wait for phase `parity` of an mbarrier: at most `limit` polls.
// Returns false on timeout.  Pipeline waits take the plan's bound
// (TileParams::wait_iters); the waits that let issued copies land before a
// timed-out CTA exits keep the default.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = kWaitIters) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Accumulator (window word) and output element of a kind.  Float pairs keep
// two float accumulators (samples u and u + 32 H) in one 64-bit register pair.
template <int KIND>
using AccT = std::conditional_t<float_pairs(KIND), unsigned long long,
                                std::conditional_t<float_kind(KIND), float, uint32_t>>;
template <int KIND>
using OutT = std::conditional_t<float_kind(KIND), float, int32_t>;

__device__ __forceinline__ uint32_t byte_sum4(uint32_t w) { return __dp4a(w, 0x01010101u, 0u); }
__device__ __forceinline__ uint32_t half_sum2(uint32_t w) { return (w & 0xffffu) + (w >> 16); }

// Unpack raw bytes into four window words (unit q of one channel).  At bin b
// each word is the sum of b consecutive raw samples (the decimated sample).
template <int KIND, int PAIR>
__device__ __forceinline__ uint4 unpack_unit(const uint8_t* raw_ch, int q, int bin) {
  uint4 v;
  if constexpr (KIND == kU8) {
    // Word k packs X[k] and X[k + PAIR] in its 16-bit lanes (bin 1 only).
    const uint32_t a = *reinterpret_cast<const uint32_t*>(raw_ch + 4 * q);
    const uint32_t b = *reinterpret_cast<const uint32_t*>(raw_ch + 4 * q + PAIR);
    const uint32_t t01 = __byte_perm(a, b, 0x5140);
    const uint32_t t23 = __byte_perm(a, b, 0x7362);
    v.x = __byte_perm(t01, 0u, 0x4140);
    v.y = __byte_perm(t01, 0u, 0x4342);
    v.z = __byte_perm(t23, 0u, 0x4140);
    v.w = __byte_perm(t23, 0u, 0x4342);
  } else if constexpr (KIND == kU4) {
    // 4-bit samples, two per byte (the earlier in the low nibble).  Word k
    // packs decimated samples k and k + PAIR in its 16-bit lanes; at bin b a
    // decimated sample is the sum of b nibbles (at most 15 * 16 = 240).
    auto nib2 = [](uint32_t w) { return (w & 0x0f0f0f0fu) + ((w >> 4) & 0x0f0f0f0fu); };
    const uint8_t* lo = raw_ch + 2 * q * bin;
    const uint8_t* hi = lo + PAIR * bin / 2;
    if (bin == 1) {
      const uint32_t c = *reinterpret_cast<const uint16_t*>(lo) |
                         (static_cast<uint32_t>(*reinterpret_cast<const uint16_t*>(hi)) << 16);
      v = make_uint4(c & 0x000f000fu, (c >> 4) & 0x000f000fu, (c >> 8) & 0x000f000fu,
                     (c >> 12) & 0x000f000fu);
    } else if (bin == 2) {  // one byte per decimated sample
      const uint32_t a = nib2(*reinterpret_cast<const uint32_t*>(lo));
      const uint32_t b = nib2(*reinterpret_cast<const uint32_t*>(hi));
      const uint32_t t01 = __byte_perm(a, b, 0x5140);
      const uint32_t t23 = __byte_perm(a, b, 0x7362);
      v = make_uint4(__byte_perm(t01, 0u, 0x4140), __byte_perm(t01, 0u, 0x4342),
                     __byte_perm(t23, 0u, 0x4140), __byte_perm(t23, 0u, 0x4342));
    } else if (bin == 4) {  // two bytes per decimated sample
      auto half = [&](uint32_t w) {
        const uint32_t s2 = nib2(w);
        return (s2 & 0x00ff00ffu) + ((s2 >> 8) & 0x00ff00ffu);
      };
      const uint2 a = *reinterpret_cast<const uint2*>(lo);
      const uint2 b = *reinterpret_cast<const uint2*>(hi);
      const uint32_t l0 = half(a.x), l1 = half(a.y), h0 = half(b.x), h1 = half(b.y);
      v = make_uint4(__byte_perm(l0, h0, 0x5410), __byte_perm(l0, h0, 0x7632),
                     __byte_perm(l1, h1, 0x5410), __byte_perm(l1, h1, 0x7632));
    } else {  // bin 8 or 16: bin / 2 bytes per decimated sample
      const int words = bin / 8;
      uint32_t o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t sl = 0, sh = 0;
        for (int j = 0; j < words; ++j) {
          sl += byte_sum4(nib2(reinterpret_cast<const uint32_t*>(lo)[k * words + j]));
          sh += byte_sum4(nib2(reinterpret_cast<const uint32_t*>(hi)[k * words + j]));
        }
        o[k] = sl | (sh << 16);
      }
      v = make_uint4(o[0], o[1], o[2], o[3]);
    }
  } else if constexpr (KIND == kU8W) {
    const uint8_t* r = raw_ch + 4 * q * bin;
    if (bin == 2) {
      const uint2 a = *reinterpret_cast<const uint2*>(r);
      const uint32_t s0 = (a.x & 0x00ff00ffu) + ((a.x >> 8) & 0x00ff00ffu);
      const uint32_t s1 = (a.y & 0x00ff00ffu) + ((a.y >> 8) & 0x00ff00ffu);
      v = make_uint4(s0 & 0xffffu, s0 >> 16, s1 & 0xffffu, s1 >> 16);
    } else if (bin == 4) {
      const uint4 a = *reinterpret_cast<const uint4*>(r);
      v = make_uint4(byte_sum4(a.x), byte_sum4(a.y), byte_sum4(a.z), byte_sum4(a.w));
    } else if (bin == 8) {
      const uint4 a = *reinterpret_cast<const uint4*>(r);
      const uint4 b = *reinterpret_cast<const uint4*>(r + 16);
      v = make_uint4(byte_sum4(a.x) + byte_sum4(a.y), byte_sum4(a.z) + byte_sum4(a.w),
                     byte_sum4(b.x) + byte_sum4(b.y), byte_sum4(b.z) + byte_sum4(b.w));
    } else {  // bin 16
      uint32_t o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint4 a = *reinterpret_cast<const uint4*>(r + 16 * k);
        o[k] = byte_sum4(a.x) + byte_sum4(a.y) + byte_sum4(a.z) + byte_sum4(a.w);
      }
      v = make_uint4(o[0], o[1], o[2], o[3]);
    }
  } else if constexpr (KIND == kU16) {
    const uint8_t* r = raw_ch + 8 * q * bin;
    if (bin == 1) {
      const uint2 a = *reinterpret_cast<const uint2*>(r);
      v = make_uint4(a.x & 0xffffu, a.x >> 16, a.y & 0xffffu, a.y >> 16);
    } else if (bin == 2) {
      const uint4 a = *reinterpret_cast<const uint4*>(r);
      v = make_uint4(half_sum2(a.x), half_sum2(a.y), half_sum2(a.z), half_sum2(a.w));
    } else {  // bin 4 or 8: bin / 2 words of two samples per output word
      uint32_t o[4];
      const int words = bin / 2;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t acc = 0;
        for (int j = 0; j < words; ++j)
          acc += half_sum2(*reinterpret_cast<const uint32_t*>(r + 4 * (k * words + j)));
        o[k] = acc;
      }
      v = make_uint4(o[0], o[1], o[2], o[3]);
    }
  } else {  // kF32
    const float* r = reinterpret_cast<const float*>(raw_ch + 16 * q * bin);
    if (bin == 1) {
      v = *reinterpret_cast<const uint4*>(r);
    } else {
      float o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float acc = 0.f;
        for (int j = 0; j < bin; ++j) acc += r[k * bin + j];
        o[k] = acc;
      }
      v = make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]),
                     __float_as_uint(o[3]));
    }
  }
  return v;
}

// Issue the TMA copies of channel stage `st` into buffer `buf` (mbarrier at
// bar_base + 8 buf).  Threads 0..NC-1 copy one channel's raw window each: it
// starts at the 16-byte aligned decimated sample at or before t0 + base and is
// clipped at the end of the row.  Thread NC copies rec_bytes of the stage's
// records from rec_src to rec_dst.  Nothing is issued (and nobody arrives)
// for the stage p.hold_stage, so the wait on it runs out: the hook that tests
// the timeout path.
template <int KIND, int NC>
__device__ __forceinline__ void issue_stage(const TileParams& p, uint32_t bar_base, uint8_t* raw,
                                            int st, int buf, int64_t t0, int32_t base, int tid,
                                            const void* rec_src, uint32_t rec_bytes,
                                            void* rec_dst) {
  if (st == p.hold_stage) return;
  const uint32_t bar = bar_base + 8u * buf;
  if (tid < NC) {
    const int c = st * NC + tid;
    uint32_t bytes = 0;
    const uint8_t* src = nullptr;
    if (c < p.n_chan) {
      // Window start: the planner's alignment (a power of two, decimated
      // samples, a multiple of the 16 bytes a copy starts on), as raw
      // samples from element 0 of the row.
      const int64_t align = p.align;
      const int64_t ua = ((t0 + base) & ~(align - 1)) * p.bin - p.x_origin;
      if (ua >= 0 && ua < p.stride) {
        const int64_t room = sample_bytes(KIND, p.stride - ua);
        bytes = static_cast<uint32_t>(room < p.lraw ? room : p.lraw);
        src = static_cast<const uint8_t*>(p.x) +
              sample_bytes(KIND, static_cast<int64_t>(c) * p.stride + ua);
      }
    }
    mbar_arrive_expect(bar, bytes);
    if (bytes) {
      uint8_t* dst = raw + (static_cast<size_t>(buf) * NC + tid) * p.lraw;
      bulk_copy(smem_u32(dst), src, bytes, bar);
    }
  } else if (tid == NC) {
    mbar_arrive_expect(bar, rec_bytes);
    bulk_copy(smem_u32(rec_dst), rec_src, rec_bytes, bar);
  }
}

// Per-channel records of stage st (Rec or PRec, base shift first): the copy
// arguments of issue_stage.
template <int NC, typename RecT>
struct ChannelRecs {
  const RecT* blk_recs;  // the block's records in global memory
  RecT* sm;              // [2][NC] in shared memory
  int n_chan;
  __device__ const void* src(int st) const { return blk_recs + st * NC; }
  __device__ uint32_t bytes(int st) const {
    return static_cast<uint32_t>(min(NC, n_chan - st * NC)) * sizeof(RecT);
  }
  __device__ void* dst(int buf) const { return sm + buf * NC; }
};

// Fire-and-forget integer add into global memory (performed at L2).
__device__ __forceinline__ void red_add(int32_t* p, int32_t v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add(float* p, float v) { atomicAdd(p, v); }
// Two adjacent int32 outputs (8-byte aligned) in one 64-bit reduction: exact
// while both are non-negative sums below 2^32 (no carry crosses the halves).
__device__ __forceinline__ void red_add_pair(int32_t* p, uint32_t lo, uint32_t hi) {
  const unsigned long long v = static_cast<unsigned long long>(hi) << 32 | lo;
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Transposed store tile of a register tile with H window words per lane.
// Lane l holds positions p = H l + j (j < H); uint8 at bin 1 also holds
// p + 32 H in the upper 16-bit halves.  The tile is read back row by row
// (p = 32 k + l).  With H odd the identity index is conflict-free for both;
// with H = 20 the index f(p) = p + p / 160 is.
template <int KIND, int H>
struct StoreTile {
  static_assert(H % 2 == 1 || H == 20, "transpose index defined for odd H and H = 20");
  static constexpr bool kPad = H % 2 == 0;
  static constexpr int kRows = H * samples_per_word(KIND);  // rows of 32 positions
  static constexpr int kPairW = 32 * H;                      // uint8 pair distance
  static constexpr int kWords =                              // per-warp tile
      kPad ? flush_words(KIND) : 32 * kRows;
  __device__ static constexpr int row(int k) { return 32 * k + (kPad ? k / 5 : 0); }
};

// Store (first) or add (later) the accumulators of DR DMs x H words per lane
// into the output rows through the warp's transposed shared tile.  The tiles
// live in the window buffer pw; when it cannot hold one per warp, the warps
// take turns in `groups` rounds.  Called by every thread of the CTA.
template <int KIND, int DR, int NW, int NC, int H, bool kPackedTile = true>
__device__ __forceinline__ void widen_store(const TileParams& p, uint32_t* pw,
                                            AccT<KIND> (&acc)[DR][H], int blk, int64_t t0,
                                            bool first) {
  using ST = StoreTile<KIND, H>;
  constexpr int kFw = ST::kWords;
  constexpr int kWw = word_bytes(KIND) / 4;  // 32-bit words per window word
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  // Window buffers hold at least 32 H + 16 window words per channel.
  constexpr bool kAllFit = NC * (32 * H + 16) * kWw >= NW * kFw;
  const int fit = (NC * p.lp * kWw) / kFw;  // tiles that fit the window buffer
  const int groups = kAllFit ? 1 : (NW + fit - 1) / fit;
  uint32_t* tr = pw + (w / groups) * kFw;
  const int wbase = H * l + (ST::kPad ? (l >> 3) : 0);
  constexpr int kHiOff = ST::kPairW + (ST::kPad ? ST::kPairW / 160 : 0);
  const int64_t lim = p.t_end - t0;
  for (int gi = 0; gi < groups; ++gi) {
    if (gi > 0) __syncthreads();
    if (w % groups != gi) continue;
#pragma unroll
    for (int i = 0; i < DR; ++i) {
      const int d = blk * (DR * NW) + w * DR + i;
      if constexpr (kPackedTile && (KIND == kU8 || KIND == kU8P) && !ST::kPad) {
        // uint8 pairs (widened every 256 channels), row 8-byte aligned:
        // packed words: the tile keeps each accumulator
        // word whole (position p and p + 32H in its halves) and lane l takes
        // words 64 m + 2 l and + 1, i.e. output pairs (p, p + 1) and
        // (p + 32H, p + 32H + 1): one 64-bit store or reduction each.
        OutT<KIND>* row = static_cast<OutT<KIND>*>(p.out) + static_cast<int64_t>(d) * p.out_stride + t0;
        if ((reinterpret_cast<uintptr_t>(row) & 7u) == 0) {
#pragma unroll
          for (int j = 0; j < H; ++j) {
            tr[wbase + j] = acc[i][j];
            acc[i][j] = 0u;
          }
          __syncwarp();
          if (d < p.n_dm) {
            auto put = [&](int pos, uint32_t a, uint32_t b) {
              if (pos + 1 < lim) {
                if (first) *reinterpret_cast<int2*>(row + pos) = make_int2(a, b);
                else red_add_pair(row + pos, a, b);
              } else if (pos < lim) {
                if (first) row[pos] = static_cast<int32_t>(a);
                else red_add(row + pos, static_cast<int32_t>(a));
              }
            };
#pragma unroll
            for (int m = 0; m < (ST::kPairW + 63) / 64; ++m) {
              const int p0 = 64 * m + 2 * l;
              if (p0 >= ST::kPairW) continue;
              const uint2 v = *reinterpret_cast<const uint2*>(tr + p0);
              put(p0, v.x & 0xffffu, v.y & 0xffffu);
              put(p0 + ST::kPairW, v.x >> 16, v.y >> 16);
            }
          }
          __syncwarp();
          continue;
        }
      }
#pragma unroll
      for (int j = 0; j < H; ++j) {
        if constexpr (packed_pairs(KIND)) {
          const uint32_t v = acc[i][j];
          tr[wbase + j] = v & 0xffffu;
          tr[wbase + j + kHiOff] = v >> 16;
          acc[i][j] = 0u;
        } else if constexpr (float_pairs(KIND)) {
          // Low float: position H l + j; high float: that + 32 H.
          tr[wbase + j] = static_cast<uint32_t>(acc[i][j]);
          tr[wbase + j + kHiOff] = static_cast<uint32_t>(acc[i][j] >> 32);
          acc[i][j] = 0ull;
        } else if constexpr (KIND == kU16 || KIND == kU8W || KIND == kU16P) {
          tr[wbase + j] = acc[i][j];
          acc[i][j] = 0u;
        } else {
          tr[wbase + j] = __float_as_uint(acc[i][j]);
          acc[i][j] = 0.f;
        }
      }
      __syncwarp();
      bool paired = false;
      if constexpr (!ST::kPad && !float_kind(KIND)) {
        // Later widenings of integer sums (non-negative) with the row 8-byte
        // aligned: lane l adds positions 64 m + 2 l and + 1 in one 64-bit
        // reduction (the tile holds position p at index p).
        OutT<KIND>* row = static_cast<OutT<KIND>*>(p.out) + static_cast<int64_t>(d) * p.out_stride + t0;
        if (!first && d < p.n_dm && (reinterpret_cast<uintptr_t>(row) & 7u) == 0) {
          constexpr int kPos = 32 * ST::kRows;
#pragma unroll
          for (int m = 0; m < (kPos + 63) / 64; ++m) {
            const int pos = 64 * m + 2 * l;
            if (pos >= kPos || pos >= lim) continue;
            const uint2 v = *reinterpret_cast<const uint2*>(tr + pos);
            if (pos + 1 < lim) red_add_pair(row + pos, v.x, v.y);
            else red_add(row + pos, static_cast<int32_t>(v.x));
          }
          paired = true;
        }
      }
      if (d < p.n_dm && !paired) {
        OutT<KIND>* row = static_cast<OutT<KIND>*>(p.out) + static_cast<int64_t>(d) * p.out_stride + t0;
        constexpr int kCh = (ST::kRows + 1) / 2;  // rows per half
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          OutT<KIND> v[kCh];
#pragma unroll
          for (int k = 0; k < kCh; ++k) {
            const int kk = h * kCh + k;
            if (kk < ST::kRows) {
              const uint32_t bits = tr[ST::row(kk) + l];
              if constexpr (float_kind(KIND)) v[k] = __uint_as_float(bits);
              else v[k] = static_cast<int32_t>(bits);
            } else {
              v[k] = OutT<KIND>(0);
            }
          }
          if (!first && !float_kind(KIND)) {
            // Later widenings of integer sums: reductions at L2 (exact, any
            // order), so the warp does not wait for the row to come back.
#pragma unroll
            for (int k = 0; k < kCh; ++k) {
              const int kk = h * kCh + k;
              const int pos = 32 * kk + l;
              if (kk < ST::kRows && pos < lim) red_add(row + pos, v[k]);
            }
            continue;
          }
          if (!first) {
            OutT<KIND> g[kCh];
#pragma unroll
            for (int k = 0; k < kCh; ++k) {
              const int kk = h * kCh + k;
              const int pos = 32 * kk + l;
              g[k] = (kk < ST::kRows && pos < lim) ? __ldcg(row + pos) : OutT<KIND>(0);
            }
#pragma unroll
            for (int k = 0; k < kCh; ++k) v[k] += g[k];
          }
#pragma unroll
          for (int k = 0; k < kCh; ++k) {
            const int kk = h * kCh + k;
            const int pos = 32 * kk + l;
            if (kk < ST::kRows && pos < lim) row[pos] = v[k];
          }
        }
      }
      __syncwarp();
    }
  }
}


// Widening slots (TileParams::wslots): one slot per CTA and unit, acquired
// from the plan's flags by thread 0 (the SM id is the first probe), released
// after the unit's last reads of it.  Returns -1 if every slot stayed held
// through the probes (the unit then reports kErrTimeout).
__device__ __forceinline__ int acquire_wslot(const TileParams& p) {
  unsigned smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  for (int probe = 0; probe < 4 * p.n_wslots; ++probe) {
    const int s = static_cast<int>((smid + static_cast<unsigned>(probe)) %
                                   static_cast<unsigned>(p.n_wslots));
    if (atomicCAS(p.wflags + s, 0, 1) == 0) {
      __threadfence();  // the slot's earlier holder is done with it
      return s;
    }
  }
  return -1;
}
__device__ __forceinline__ void release_wslot(const TileParams& p, int slot) {
  __threadfence();
  atomicExch(p.wflags + slot, 0);
}

// One warp widens its 16-bit lanes into its part of the slot: accumulator
// word (i, j) of lane l (samples at positions H l + j and H l + j + 32 H)
// adds its halves into 64-bit word (i H + j) 32 + l as two 32-bit sums (each
// below 2^32: no carry crosses them).  The first widening of a unit stores.
// Lanes are zeroed.  Coalesced: a warp's 32 words are 256 contiguous bytes.
template <int DR, int H>
__device__ __forceinline__ void widen_to_slot(unsigned long long* warp_slot,
                                              uint32_t (&acc)[DR][H], bool first) {
  const int l = threadIdx.x & 31;
  unsigned long long* q = warp_slot + l;
#pragma unroll
  for (int i = 0; i < DR; ++i)
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const uint32_t a = acc[i][j];
      const unsigned long long v =
          static_cast<unsigned long long>(a & 0xffffu) |
          static_cast<unsigned long long>(a >> 16) << 32;
      unsigned long long* w = q + (i * H + j) * 32;
      if (first)
        asm volatile("st.global.u64 [%0], %1;" ::"l"(w), "l"(v) : "memory");
      else
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(w), "l"(v) : "memory");
      acc[i][j] = 0u;
    }
}

// Widening by phases: word k = i H + j of the lanes belongs to phase k mod G;
// at the end of stage st a warp widens the words of phase st mod G only, so
// each word is widened every G stages (G NC channels, within the lanes'
// bound when G NC <= the flush interval) and a stage carries 1 / G of the
// widening instead of every G-th stage all of it.  Stores in the first G
// stages (each word's first widening), reductions after.
template <int DR, int H, int G, int C>
__device__ __forceinline__ void widen_words(unsigned long long* q, uint32_t (&acc)[DR][H],
                                            bool first) {
#pragma unroll
  for (int k = C; k < DR * H; k += G) {
    const int i = k / H, j = k % H;
    const uint32_t a = acc[i][j];
    const unsigned long long v = static_cast<unsigned long long>(a & 0xffffu) |
                                 static_cast<unsigned long long>(a >> 16) << 32;
    unsigned long long* w = q + k * 32;
    if (first)
      asm volatile("st.global.u64 [%0], %1;" ::"l"(w), "l"(v) : "memory");
    else
      asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(w), "l"(v) : "memory");
    acc[i][j] = 0u;
  }
}
template <int DR, int H, int G>
__device__ __forceinline__ void widen_phase(unsigned long long* warp_slot,
                                            uint32_t (&acc)[DR][H], int phase, bool first) {
  static_assert(G == 2 || G == 4 || G == 8, "phases are generated for G = 2, 4, 8");
  unsigned long long* q = warp_slot + (threadIdx.x & 31);
  if constexpr (G == 2) {
    if (phase == 0) widen_words<DR, H, G, 0>(q, acc, first);
    else widen_words<DR, H, G, 1>(q, acc, first);
  } else if constexpr (G == 4) {
    switch (phase) {
      case 0: widen_words<DR, H, G, 0>(q, acc, first); break;
      case 1: widen_words<DR, H, G, 1>(q, acc, first); break;
      case 2: widen_words<DR, H, G, 2>(q, acc, first); break;
      default: widen_words<DR, H, G, 3>(q, acc, first); break;
    }
  } else {
    switch (phase) {
      case 0: widen_words<DR, H, G, 0>(q, acc, first); break;
      case 1: widen_words<DR, H, G, 1>(q, acc, first); break;
      case 2: widen_words<DR, H, G, 2>(q, acc, first); break;
      case 3: widen_words<DR, H, G, 3>(q, acc, first); break;
      case 4: widen_words<DR, H, G, 4>(q, acc, first); break;
      case 5: widen_words<DR, H, G, 5>(q, acc, first); break;
      case 6: widen_words<DR, H, G, 6>(q, acc, first); break;
      default: widen_words<DR, H, G, 7>(q, acc, first); break;
    }
  }
}

// The unit's outputs from a slot: each warp adds its lanes to the sums its
// earlier widenings left in its part of the slot (for word k = i H + j only
// if k mod G < done: the phases widened at least once; G = 1 with done = 0
// or 1 when every word is widened together), writes
// the 32-bit totals of its DMs into its transposed shared tile (position
// H l + j and that + 32 H, as widen_store) and stores every output row of the
// tile once.  Called by every thread of the CTA (the tiles take turns in
// `groups` rounds when the window buffer cannot hold one per warp).
template <int KIND, int DR, int NW, int NC, int H>
__device__ __forceinline__ void store_from_slot(const TileParams& p, uint32_t* pw,
                                                uint32_t (&acc)[DR][H],
                                                const unsigned long long* warp_slot, int G,
                                                int done, int blk, int64_t t0) {
  static_assert(H % 2 == 1, "the transposed tile needs an odd lane stride");
  constexpr int kPairW = 32 * H;
  constexpr int kRows = 2 * H;            // rows of 32 positions
  constexpr int kFw = 32 * kRows;         // per-warp tile
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  constexpr bool kAllFit = NC * (32 * H + 16) >= NW * kFw;
  const int fit = (NC * p.lp) / kFw;
  const int groups = kAllFit ? 1 : (NW + fit - 1) / fit;
  uint32_t* tr = pw + (w / groups) * kFw;
  const int wbase = H * l;
  const int64_t lim = p.t_end - t0;
  // This thread's reductions into its words of the slot are performed before
  // it reads them back.
  if (done > 0) __threadfence();
  for (int gi = 0; gi < groups; ++gi) {
    if (gi > 0) __syncthreads();
    if (w % groups != gi) continue;
#pragma unroll
    for (int i = 0; i < DR; ++i) {
      const int d = blk * (DR * NW) + w * DR + i;
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const uint32_t a = acc[i][j];
        uint32_t lo = a & 0xffffu, hi = a >> 16;
        if ((i * H + j) % G < done) {
          const unsigned long long v = __ldcg(warp_slot + (i * H + j) * 32 + l);
          lo += static_cast<uint32_t>(v);
          hi += static_cast<uint32_t>(v >> 32);
        }
        tr[wbase + j] = lo;
        tr[wbase + j + kPairW] = hi;
        acc[i][j] = 0u;
      }
      __syncwarp();
      if (d < p.n_dm) {
        OutT<KIND>* row =
            static_cast<OutT<KIND>*>(p.out) + static_cast<int64_t>(d) * p.out_stride + t0;
#pragma unroll 4
        for (int k = 0; k < kRows; ++k) {
          const int pos = 32 * k + l;
          if (pos < lim) row[pos] = static_cast<int32_t>(tr[pos]);
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace tk
}  // namespace dd
