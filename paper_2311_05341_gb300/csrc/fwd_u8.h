// fwd_u8.h -- geometry, device table record and launch parameters of the
// register-tiled uint8 kernel (fwd_u8.cu), shared with the planner.
#pragma once

#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define DD_HOST_DEVICE __host__ __device__
#else
#define DD_HOST_DEVICE
#endif

namespace dd {
namespace u8k {

constexpr int kH = 20;               // paired words per lane per DM (40 samples)
constexpr int kPair = 32 * kH;       // word u packs samples u and u + kPair
constexpr int kTile = 2 * kPair;     // output samples per CTA
constexpr int kMaxOff = 15;          // largest in-window DM offset (4-bit field)
constexpr int kWin = 36;             // window words per lane (>= kH + kMaxOff, multiple of 4)
constexpr int kFlushChannels = 256;  // 255 * 256 < 2^16: widen before lanes overflow
constexpr int kFlushWords = 1288;    // per-warp transpose tile (1280 + 1280/160 pad)
constexpr int kMaxWarps = 12;
constexpr int kWaitIters = 1 << 22;  // bound on every mbarrier wait loop
constexpr int kErrTimeout = 1;       // device status bit: a bounded wait gave up
constexpr size_t kStatusOffset = 0;  // status word at the start of the plan workspace
constexpr size_t kStatusBytes = 256;

// Tile shapes: DMs per warp (the register tile is dr DMs x 40 samples per
// lane), warps per CTA, CTAs per SM and channels per pipeline stage.  Fewer DMs
// per lane free registers for more resident warps (latency hiding) at the cost
// of more shared-memory traffic per add; the autotuner picks per plan.
struct Shape {
  int dr;
  int warps;
  int min_blocks;
  int nc;
};
constexpr Shape kShapes[] = {{8, 8, 1, 16}, {6, 12, 1, 24}, {4, 8, 2, 16}};
constexpr int kNumShapes = 3;

inline const Shape* shape_for(int dr) {
  for (const Shape& s : kShapes)
    if (s.dr == dr) return &s;
  return nullptr;
}

// Per (DM block of dr * warps DMs, channel) record, 64 bytes (TMA-copyable).
struct Rec {
  int32_t base;               // s(c, first DM of the block)
  uint32_t delta[kMaxWarps];  // dr x 4-bit in-window offsets of warp w's DMs
  uint8_t aq[kMaxWarps];      // warp w's window start, in 16-byte units
};
static_assert(sizeof(Rec) == 64, "Rec must stay 64 bytes");

constexpr size_t kRecOffset = 128;
DD_HOST_DEVICE constexpr size_t raw_offset(int nc) {
  const size_t end = kRecOffset + 2 * static_cast<size_t>(nc) * sizeof(Rec);
  return (end + 127) / 128 * 128;
}

// Words of a channel's paired window for a given DM-block shift span.
inline int32_t window_words(int32_t span) {
  const int32_t need = kH * 31 + (span + 15) + kWin;  // last lane, widest offset
  return (need + 15) / 16 * 16;
}

inline size_t smem_bytes(const Shape& s, int32_t lp) {
  return raw_offset(s.nc) + 2 * static_cast<size_t>(s.nc) * (lp + kPair) +
         static_cast<size_t>(s.nc) * lp * 4;
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
  uint32_t units_magic; // u / (lp/4) == (u * magic) >> (32 + shift)
  int32_t units_shift;
  int32_t* out;
  int32_t* err;
};

}  // namespace u8k
}  // namespace dd
