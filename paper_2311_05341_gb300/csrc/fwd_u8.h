// fwd_u8.h -- geometry, device table record and launch parameters of the
// register-tiled uint8 kernel (fwd_u8.cu), shared with the planner.
#pragma once

#include <cstddef>
#include <cstdint>

namespace dd {
namespace u8k {

constexpr int kH = 20;               // paired words per lane per DM (40 samples)
constexpr int kDR = 8;               // DMs per warp (and per lane)
constexpr int kWarps = 8;            // warps per CTA
constexpr int kThreads = 32 * kWarps;
constexpr int kPair = 32 * kH;       // word u packs samples u and u + kPair
constexpr int kTile = 2 * kPair;     // output samples per CTA
constexpr int kDmCta = kDR * kWarps; // DMs per CTA
constexpr int kNC = 16;              // channels per pipeline stage
constexpr int kMaxOff = 15;          // largest in-window DM offset (4-bit field)
constexpr int kWin = 36;             // window words per lane (>= kH + kMaxOff, multiple of 4)
constexpr int kFlushChannels = 256;  // 255 * 256 < 2^16: widen before lanes overflow
constexpr int kFlushWords = 1288;    // per-warp transpose tile (1280 + 1280/160 pad)
constexpr int kWaitIters = 1 << 22;  // bound on every mbarrier wait loop
constexpr int kErrTimeout = 1;       // device status bit: a bounded wait gave up
constexpr size_t kStatusOffset = 0;  // status word at the start of the plan workspace
constexpr size_t kStatusBytes = 256;

// Per (DM block of kDmCta, channel) record, 48 bytes (TMA-copyable).
struct Rec {
  int32_t base;            // s(c, first DM of the block)
  uint32_t delta[kWarps];  // 8 x 4-bit in-window offsets of warp w's DMs
  uint8_t aq[kWarps];      // warp w's window start, in 16-byte units
  uint8_t pad[4];
};
static_assert(sizeof(Rec) == 48, "Rec must stay 48 bytes");

constexpr size_t kRecOffset = 128;
constexpr size_t kRawOffset = kRecOffset + 2 * kNC * sizeof(Rec);
static_assert(kRawOffset % 128 == 0, "raw staging must stay 128-byte aligned");

// Words of a channel's paired window for a given DM-block shift span.
inline int32_t window_words(int32_t span) {
  const int32_t need = kH * 31 + (span + 15) + kWin;  // last lane, widest offset
  return (need + 15) / 16 * 16;
}

inline size_t smem_bytes(int32_t lp) {
  return kRawOffset + 2 * static_cast<size_t>(kNC) * (lp + kPair) +
         static_cast<size_t>(kNC) * lp * 4;
}

struct U8Params {
  const uint8_t* x;
  int64_t stride;       // bytes between channel rows
  int32_t n_chan;
  const Rec* recs;      // [n_blocks][n_chan]
  int32_t n_dm;
  int32_t n_blocks;
  int64_t n_out;
  int32_t lp;           // paired words per staged channel window
  int32_t lraw;         // raw bytes per staged channel window (lp + kPair)
  uint32_t units_magic; // u / (lp/4) == umulhi(u, magic) >> shift
  int32_t units_shift;
  int32_t* out;
  int32_t* err;
};

}  // namespace u8k
}  // namespace dd
