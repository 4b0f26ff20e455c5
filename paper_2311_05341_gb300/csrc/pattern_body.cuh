// pattern_body.cuh -- device code of the pattern tiles (fwd_pattern.cu): the
// shared-memory layout, the generated pattern blocks and the (DM block, time
// tile) work unit, shared by the one-unit-per-CTA kernel and the persistent
// batch kernel (fwd_pattern_batch.cu).
//
// Computes Eq. 3 (Algorithm 1) with the output partition, staging and
// binning of the offset tiles (fwd_tiled.cu); the register tile, its
// per-channel dispatch and the widening of 16-bit lanes into per-CTA slots
// differ:
//
//  * Every lane owns kPatDr = 4 consecutive DMs x H window words, H odd
//    (uint8: 2H samples, pairing samples u and u + 32H in 16-bit lanes).
//  * Eq. 1 is linear in DM, so from one trial DM to the next the shift of a
//    channel grows by the floor or the ceiling of step * k_c / (bin * t_samp):
//    the increments between a warp's four DMs are a or a + 1.  The host
//    stores, per (DM block, channel, warp), the window offset of the warp's
//    first DM and the pattern 8 a + bits (fwd_tiled.h).
//  * Integer kinds: each warp walks its own list of channel pairs that share
//    a pattern; per pair one warp-uniform indexed branch enters a generated
//    block (gen_dispatch.py) that loads the window words its offsets touch
//    (scalar shared loads, conflict-free at any offset because the lane
//    stride H is odd) and adds both channels' samples with three-input adds.
//    Float pairs: the same, the two channels' words summed once per word
//    before the four DMs add the sum.  Single floats: one channel per branch.
//  * 16-bit lanes (uint8, 4-bit) widen into a slot of the plan workspace
//    (widening modes, tk::widen_mode), or without one into the output rows.
//
// Against the 4-bit-offset tiles this is one indexed branch per four DMs and
// two channels instead of one per DM.  Every mbarrier wait is bounded; on
// timeout the unit records kErrTimeout in the status word and returns false.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fwd_tiled.h"
#include "fwd_tiled_dispatch.inc"
#include "tile_common.cuh"

namespace dd {
namespace tk {
namespace pattern {

struct PSmem {
  uint32_t bar_base;  // 2 mbarriers
  unsigned char* recs;  // [2][NC] PRec, or [2] pair chunks
  uint8_t* raw;       // [NC][lraw]
  uint32_t* pw;       // [1 or 2][NC][lp] window words
};

template <int NW, int NC, bool PAIRS, bool DBUF>
__device__ __forceinline__ PSmem pat_layout(unsigned char* smem, int32_t lraw) {
  constexpr size_t kRawOff = pat_raw_offset(PatShape{0, NW, NC, PAIRS, DBUF, 0});
  PSmem sm;
  sm.bar_base = smem_u32(smem);
  sm.recs = smem + kRecOffset;
  sm.raw = smem + kRawOff;
  sm.pw = reinterpret_cast<uint32_t*>(sm.raw + NC * static_cast<size_t>(lraw));
  return sm;
}

// One channel (or a pair of channels of one pattern) into the lane's
// accumulators: `win` (`win2`) is the shared-memory address of the lane's
// window; the generated block of pattern `ix` loads the window words it needs
// and adds them.  The blocks exist for the window widths gen_dispatch.py lists.
template <int KIND, int H>
__device__ __forceinline__ void pat_channel(AccT<KIND> (&acc)[kPatDr][H], uint32_t win,
                                            uint32_t ix) {
  if constexpr (float_pairs(KIND)) {
    static_assert(H == 11 || H == 13, "no generated float-pair blocks for H");
    if constexpr (H == 11) DD_PATL_CHANNEL_F2_11(acc, win, ix);
    else DD_PATL_CHANNEL_F2_13(acc, win, ix);
    return;
  } else {
  static_assert(H == 15 || H == 17 || H == 19 || H == 21 || H == 23 || H == 25,
                "no generated pattern blocks for H");
#define DD_PAT_CASE(HH)                                                  \
  if constexpr (H == HH) {                                               \
    if constexpr (float_kind(KIND)) DD_PATL_CHANNEL_F32_##HH(acc, win, ix);  \
    else DD_PATL_CHANNEL_U32_##HH(acc, win, ix);                         \
  }
  DD_PAT_CASE(15)
  DD_PAT_CASE(17)
  DD_PAT_CASE(19)
  DD_PAT_CASE(21)
  DD_PAT_CASE(23)
  DD_PAT_CASE(25)
#undef DD_PAT_CASE
  }
}

// The same with the window words already in registers R (H + 6 of them): the
// loads are scheduled before the branch.  Single-channel tiles run faster so.
template <int KIND, int H>
__device__ __forceinline__ void pat_channel_regs(AccT<KIND> (&acc)[kPatDr][H],
                                                 const AccT<KIND> (&R)[H + 2 * (kPatDr - 1)],
                                                 uint32_t ix) {
#define DD_PAT_CASE(HH)                                           \
  if constexpr (H == HH) {                                        \
    if constexpr (float_kind(KIND)) DD_PAT_CHANNEL_F32_##HH(acc, R, ix); \
    else DD_PAT_CHANNEL_U32_##HH(acc, R, ix);                     \
  }
  DD_PAT_CASE(15)
  DD_PAT_CASE(17)
  DD_PAT_CASE(19)
  DD_PAT_CASE(21)
  DD_PAT_CASE(23)
  DD_PAT_CASE(25)
#undef DD_PAT_CASE
}

template <int KIND, int H>
__device__ __forceinline__ void pat_pair(AccT<KIND> (&acc)[kPatDr][H], uint32_t win,
                                         uint32_t win2, uint32_t ix) {
  if constexpr (float_pairs(KIND)) {
    static_assert(H == 11 || H == 13, "no generated float-pair pair blocks for H");
    if constexpr (H == 11) DD_PATL2_CHANNEL_F2_11(acc, win, win2, ix);
    else DD_PATL2_CHANNEL_F2_13(acc, win, win2, ix);
    return;
  } else {
  static_assert(H == 15 || H == 17 || H == 19 || H == 21 || H == 23 || H == 25,
                "no generated pair blocks for H");
  // Packed uint8 / 4-bit copies take the blocks that load 7 words ahead.
#define DD_PAIR_CASE(HH)                                                         \
  if constexpr (H == HH) {                                                       \
    if constexpr (KIND == kU8P) DD_PATL2_CHANNEL_U32P_##HH(acc, win, win2, ix);  \
    else DD_PATL2_CHANNEL_U32_##HH(acc, win, win2, ix);                          \
  }
  DD_PAIR_CASE(15)
  DD_PAIR_CASE(17)
  DD_PAIR_CASE(19)
  DD_PAIR_CASE(21)
  DD_PAIR_CASE(23)
  DD_PAIR_CASE(25)
#undef DD_PAIR_CASE
  }
}

// Pair chunk of one (DM block, stage) in global memory.
__device__ __forceinline__ const unsigned char* pair_chunk(const TileParams& p, int blk, int n_st,
                                                           int st) {
  return static_cast<const unsigned char*>(p.recs) +
         (static_cast<int64_t>(blk) * n_st + st) * p.chunk_bytes;
}

// One (DM block, time tile) work unit.  Returns false after a bounded wait
// gave up (the status word is set).
//
// One raw buffer: the copies of stage st + 1 are issued as soon as stage st
// is unpacked (after the barrier that follows the unpacking) and land while
// stage st is computed, so the raw bytes need no second buffer.  Records use
// two buffers (stage st in st % 2).  With DBUF the window words are
// double-buffered (stage st in window buffer st % 2) and that barrier is the
// only one per stage: it also certifies that every warp finished computing
// stage st - 1, whose window and record buffers are the next ones reused.
// Without DBUF a second barrier ends each stage.
//
// Direct kinds (packed uint8 input, float32 at bin 1) stage window words: two staging buffers
// (stage st in st % 2, each with its own mbarrier), the copies of stage st + 1
// issued at the top of stage st (its buffer was last read in stage st - 1,
// which ended with a barrier), no unpacking, and one barrier per stage (it
// also carries the bounded-wait status).
template <int KIND, int H, int NW, int NC, bool PAIRS, bool DBUF, int AMAX, int SLOTS>
__device__ __forceinline__ bool pat_body(const TileParams& p, const PSmem& sm, int blk,
                                         int64_t tile) {
  static_assert(!PAIRS || !float_kind(KIND) || float_pairs(KIND),
                "channel pairs need integer window words or float pairs");
  constexpr bool kDirect = direct_kind(KIND);
  constexpr uint32_t kWB = word_bytes(KIND);  // bytes per window word
  static_assert(!kDirect || !DBUF, "packed input stages its window words directly");
  constexpr int kPairW = 32 * H;
  constexpr int kRecBufs = 2;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int64_t t0 = tile * pat_tile_samples(KIND, H);
  const int n_st = (p.n_chan + NC - 1) / NC;

  const PRec* my_recs = static_cast<const PRec*>(p.recs) + static_cast<int64_t>(blk) * p.n_chan;
  const int32_t* my_bases = p.bases + static_cast<int64_t>(blk) * p.n_chan;
  auto base_of = [&](int st) -> int32_t {
    const int c = st * NC + tid;
    if (!(tid < NC && st < n_st && c < p.n_chan)) return 0;
    if constexpr (PAIRS) return my_bases[c];
    else return my_recs[c].base;
  };
  auto rec_buf = [&](int rb) -> unsigned char* {
    if constexpr (PAIRS) return sm.recs + rb * p.chunk_bytes;
    else return sm.recs + rb * NC * static_cast<int>(sizeof(PRec));
  };
  const ChannelRecs<NC, PRec> cr{my_recs, reinterpret_cast<PRec*>(sm.recs), p.n_chan};
  auto issue = [&](int st, int32_t base) {
    unsigned char* dst = rec_buf(st % kRecBufs);
    const int sbuf = kDirect ? (st & 1) : 0;
    if constexpr (PAIRS)
      issue_stage<KIND, NC>(p, sm.bar_base, sm.raw, st, sbuf, t0, base, tid,
                            pair_chunk(p, blk, n_st, st), p.chunk_bytes, dst);
    else
      issue_stage<KIND, NC>(p, sm.bar_base, sm.raw, st, sbuf, t0, base, tid, cr.src(st),
                            cr.bytes(st), dst);
  };
  // SLOTS (16-bit lanes, the plan's workspace has widening slots): each warp
  // widens into its part of the CTA's slot when its lanes are full, before
  // the stage barrier, with no shared-memory transpose and no barrier of its
  // own; the last stage stores each output once.  All warps widen at the
  // same stage: staggering them over the stages (two warps per stage) ran
  // 1.3 % slower, every stage then waiting at its barrier for the warps that
  // widen.  Otherwise the CTA widens into the output rows together.  The
  // slot index stays in shared memory.  The slot is taken before the unit
  // issues any copy: if none comes free within the probes (at most one CTA
  // of these tiles runs per SM and the workspace has twice as many slots as
  // a GB300 has SMs), the unit reports kErrTimeout and computes nothing.
  // SLOTS = G >= 2 widens by G phases (widen_phase: 1 / G of the words at
  // the end of every stage; the launch picks it when the lanes take exactly G
  // stages): 4 % faster on the paper plan (G = 8) than every word every 8th
  // stage (SLOTS 1), whose stage barrier waited for all warps' widenings at
  // once.
  static_assert(!SLOTS || packed_pairs(KIND), "widening slots serve 16-bit lanes");
  constexpr bool kPhased = SLOTS >= 2;
  constexpr int kPhases = kPhased ? SLOTS : 1;
  __shared__ int s_wslot;
  if constexpr (SLOTS) {
    if (tid == 0) {
      s_wslot = acquire_wslot(p);
      if (s_wslot < 0) atomicOr(p.err, kErrTimeout);
    }
    __syncthreads();
    if (s_wslot < 0) return false;
  }
  auto warp_slot = [&]() {
    return p.wslots + static_cast<int64_t>(s_wslot) * p.wslot_words +
           static_cast<int64_t>(w) * kPatDr * 32 * H;
  };
  // Timeout exit with a slot held: every thread's slot writes are ordered
  // before thread 0 frees it.
  auto drop_slot = [&]() {
    if constexpr (SLOTS) {
      __threadfence();
      __syncthreads();
      if (tid == 0) release_wslot(p, s_wslot);
    }
  };

  if (tid <= NC) {
    // Shared memory read by an earlier unit of a persistent CTA is rewritten
    // by the copies: order those generic-proxy reads before them.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(0, base_of(0));
  }
  int32_t next_base = base_of(1);
  auto issue_next = [&](int st) {  // copies of stage st + 1 once stage st is unpacked
    if (tid <= NC && st + 1 < n_st) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(st + 1, next_base);
      next_base = base_of(st + 2);
    }
  };

  AccT<KIND> acc[kPatDr][H];
#pragma unroll
  for (int i = 0; i < kPatDr; ++i)
#pragma unroll
    for (int j = 0; j < H; ++j) acc[i][j] = AccT<KIND>(0);

  bool first = true;
  int since = 0;  // channels accumulated since the last widen
  const int units = p.lp >> 2;
  int rb = 0;     // st % kRecBufs

  for (int st = 0; st < n_st; ++st) {
    const int buf = st & 1;
    // One stage barrier completes a phase per stage; with kDirect each of the
    // two completes one every other stage.
    const uint32_t parity = kDirect ? (st >> 1) & 1 : st & 1;
    const uint32_t bar = sm.bar_base + (kDirect ? 8u * buf : 0u);
    const int nc = min(NC, p.n_chan - st * NC);
    uint32_t* pwb = kDirect ? reinterpret_cast<uint32_t*>(sm.raw + static_cast<size_t>(buf) * NC * p.lraw)
                            : sm.pw + (DBUF ? static_cast<size_t>(buf) * NC * p.lp : 0);
    auto unpack = [&]() {  // raw bytes of stage st into window words
      // Warp w takes channels w, w + NW, ...; its lanes take consecutive units
      // (conflict-free 16-byte stores).
      if constexpr (!kDirect) {
        const uint8_t* rawb = sm.raw;
        for (int ch = w; ch < nc; ch += NW) {
          const uint8_t* raw_ch = rawb + static_cast<size_t>(ch) * p.lraw;
          uint32_t* dst = pwb + static_cast<size_t>(ch) * p.lp;
          for (int q = l; q < units; q += 32)
            *reinterpret_cast<uint4*>(dst + 4 * q) = unpack_unit<KIND, kPairW>(raw_ch, q, p.bin);
        }
      }
    };
    if constexpr (kDirect) issue_next(st);
    const bool ok = mbar_wait(bar, parity, p.wait_iters);
    if constexpr (!kDirect) {
      if (ok) unpack();
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(p.err, kErrTimeout);
          // Let the copies still in flight land before the CTA exits (bounded).
          if (st != p.hold_stage) mbar_wait(bar, parity);
        }
        drop_slot();
        return false;
      }
      issue_next(st);
    }

    // Shift-and-sum.  The loops stay rolled so the dispatch blocks, and their
    // PTX labels, appear once per instantiation.  A direct-kind thread whose
    // wait gave up skips it: its records may not have landed (the stage ends
    // with the barrier that reports the timeout; no barrier lies in between).
    if (kDirect && !ok) {
      // nothing to add
    } else if constexpr (PAIRS) {
      const uint32_t lane_win = smem_u32(pwb) + kWB * H * l;
      const unsigned char* ck = rec_buf(rb);
      const int n_pairs = ck[w], n_items = n_pairs + ck[kPairMaxWarps + w];
      const PairItem* items = reinterpret_cast<const PairItem*>(ck + kPairCountBytes) + w * NC;
#pragma unroll 1
      for (int k = 0; k < n_pairs; ++k) {
        const PairItem it = items[k];
        pat_pair<KIND, H>(acc, lane_win + kWB * (it.a & 0xffffu), lane_win + kWB * (it.a >> 16),
                          it.pat);
      }
#pragma unroll 1
      for (int k = n_pairs; k < n_items; ++k) {
        const PairItem it = items[k];
        pat_channel<KIND, H>(acc, lane_win + kWB * it.a, it.pat);
      }
    } else if constexpr (AMAX <= 1) {
      // Base increments 0 and 1 only: the lane's H + 6 window words are loaded
      // before the branch.
      constexpr int kR = H + 2 * (kPatDr - 1);
      const PRec* rs = reinterpret_cast<const PRec*>(rec_buf(rb));
      const uint32_t* lane_pw = pwb + H * l;
#pragma unroll 1
      for (int ch = 0; ch < nc; ++ch) {
        const uint32_t e = rs[ch].w[w];
        const uint32_t* src = lane_pw + static_cast<size_t>(ch) * p.lp + (e & kPatOffMask);
        AccT<KIND> R[kR];
#pragma unroll
        for (int k = 0; k < kR; ++k) {
          if constexpr (float_kind(KIND)) R[k] = __uint_as_float(src[k]);
          else R[k] = src[k];
        }
        pat_channel_regs<KIND, H>(acc, R, e >> kPatOffBits);
      }
    } else {
      const PRec* rs = reinterpret_cast<const PRec*>(rec_buf(rb));
      const uint32_t lane_win = smem_u32(pwb) + kWB * H * l;
#pragma unroll 1
      for (int ch = 0; ch < nc; ++ch) {
        const uint32_t e = rs[ch].w[w];
        pat_channel<KIND, H>(acc, lane_win + kWB * (ch * p.lp + (e & kPatOffMask)),
                             e >> kPatOffBits);
      }
    }
    since += nc;
    rb = rb + 1 == kRecBufs ? 0 : rb + 1;
    const bool last = st == n_st - 1;
    if constexpr (kPhased) {
      // The words of this stage's phase, before the stage barrier.
      if (!last) widen_phase<kPatDr, H, kPhases>(warp_slot(), acc, st % kPhases, st < kPhases);
    } else if constexpr (SLOTS) {
      // A warp whose lanes could not take the next stage widens into the slot
      // now, before the stage barrier (registers to global memory only).
      if (!last && since + NC > p.flush) {
        widen_to_slot<kPatDr, H>(warp_slot(), acc, first);
        first = false;
        since = 0;
      }
    }
    if constexpr (kDirect) {
      // The window words are free; a wait that gave up (its stage was added
      // from stale words, never stored) ends the unit once the copies in
      // flight have landed (bounded).
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(p.err, kErrTimeout);
          if (st != p.hold_stage) mbar_wait(bar, parity);
          if (st + 1 < n_st && st + 1 != p.hold_stage)
            mbar_wait(sm.bar_base + 8u * (buf ^ 1), ((st + 1) >> 1) & 1);
        }
        drop_slot();
        return false;
      }
    } else if constexpr (!DBUF) {
      __syncthreads();  // the window words are free
    }
    if (SLOTS ? last : since + NC > p.flush || last) {
      // The transpose tiles reuse this stage's window buffer: wait until every
      // warp has finished reading it.
      if constexpr (DBUF) __syncthreads();
      if constexpr (kPhased)
        store_from_slot<KIND, kPatDr, NW, NC, H>(p, pwb, acc, warp_slot(), kPhases,
                                                 min(kPhases, n_st - 1), blk, t0);
      else if constexpr (SLOTS)
        store_from_slot<KIND, kPatDr, NW, NC, H>(p, pwb, acc, warp_slot(), 1, first ? 0 : 1,
                                                 blk, t0);
      else
        widen_store<KIND, kPatDr, NW, NC, H>(p, pwb, acc, blk, t0, first);
      first = false;
      since = 0;
      // The next stage unpacks into this window buffer (single-buffered):
      // wait until every warp has read its transpose tile back.
      if constexpr (!DBUF) __syncthreads();
    }
  }
  if constexpr (SLOTS) {
    // Every warp has read its part of the slot back (store_from_slot).
    __threadfence();
    __syncthreads();
    if (tid == 0) release_wslot(p, s_wslot);
  }
  return true;
}

}  // namespace pattern
}  // namespace tk
}  // namespace dd
