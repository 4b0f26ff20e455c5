// fwd_tiled.h -- geometry, device table record and launch parameters of the
// register-tiled forward kernels (fwd_tiled.cu), shared with the planner and
// the batch runtime.
#pragma once

#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define DD_HOST_DEVICE __host__ __device__
#else
#define DD_HOST_DEVICE
#endif

namespace dd {
namespace tk {

// Window-word kinds of the tiled kernels: uint8 at time bin 1 and 4-bit input
// at any bin pack two (decimated) samples per 32-bit word (16-bit lanes);
// uint8 at a larger bin (kU8W), uint16 and float32 keep one (decimated) sample
// per word.  kU8P: uint8 at bin 1 read from a packed copy of the input whose
// 32-bit word t already holds samples t and t + pair in its 16-bit halves (the
// pattern tiles stage it as window words directly).  kF32D: float32 at bin 1
// staged as window words directly (the input words are the window words).
// kU16P: uint16 at bin 1 read from a copy widened to 32-bit words.  kF32P:
// float32 at bin 1 read from a packed copy of 64-bit words, word t holding
// samples t and t + pair as two floats, added two at a time (add.f32x2).
// Values 1-3 equal dd_dtype.
enum Kind : int {
  kU8 = 1, kU16 = 2, kF32 = 3, kU8W = 4, kU4 = 5, kU8P = 6, kF32D = 7, kU16P = 8, kF32P = 9
};

// Float window words; kinds whose staged words are the window words; kinds
// that read a packed copy of the input made in caller scratch.
DD_HOST_DEVICE constexpr bool float_kind(int kind) {
  return kind == kF32 || kind == kF32D || kind == kF32P;
}
DD_HOST_DEVICE constexpr bool packed_copy_kind(int kind) {
  return kind == kU8P || kind == kU16P || kind == kF32P;
}
DD_HOST_DEVICE constexpr bool direct_kind(int kind) {
  return packed_copy_kind(kind) || kind == kF32D;
}

// Window words pair samples u and u + pair in their 16-bit halves.
DD_HOST_DEVICE constexpr bool packed_pairs(int kind) {
  return kind == kU8 || kind == kU4 || kind == kU8P;
}

constexpr int kH = 20;               // window words per lane per DM (the register tile width)
constexpr int kMaxOff = 15;          // largest in-window DM offset (4-bit field)
constexpr int kWin = 36;             // window words per lane (>= kH + kMaxOff, multiple of 4)
constexpr int kPair = 32 * kH;       // uint8: word u packs samples u and u + kPair
// Per-warp transpose tile of the widen/store: 1280 (uint8 pairs) or 640
// positions plus the p / 160 padding, rounded up.
DD_HOST_DEVICE constexpr int flush_words(int kind) { return kind == 1 ? 1288 : 648; }
constexpr int kMaxWarps = 12;
constexpr int kWaitIters = 1 << 22;  // default bound on the polls of an mbarrier wait
constexpr int kErrTimeout = 1;       // device status bit: a bounded wait gave up
constexpr size_t kStatusOffset = 0;  // status word at the start of the plan workspace
constexpr size_t kStatusBytes = 256;

// Window words of two floats (samples u and u + pair), 8 bytes each.
DD_HOST_DEVICE constexpr bool float_pairs(int kind) { return kind == kF32P; }
// Bytes of one window word.
DD_HOST_DEVICE constexpr int word_bytes(int kind) { return float_pairs(kind) ? 8 : 4; }

// Samples held by one window word: two for the packed-pair kinds.
DD_HOST_DEVICE constexpr int samples_per_word(int kind) {
  return packed_pairs(kind) || float_pairs(kind) ? 2 : 1;
}
// Output samples per CTA tile: 32 lanes x kH words x samples per word.
DD_HOST_DEVICE constexpr int tile_samples(int kind) { return 32 * kH * samples_per_word(kind); }
// Bytes of one element of the rows a kind stages (kF32P: a 64-bit word of
// its packed copy).
DD_HOST_DEVICE constexpr int elem_bytes(int kind) {
  return (kind == kU8 || kind == kU8W || kind == kU4) ? 1
         : kind == kU16                              ? 2
         : kind == kF32P                             ? 8
                                                     : 4;
}
// Raw samples per 16 bytes (4-bit samples: two per byte; kU8P: positions of
// the packed copy, one 4-byte word each).
DD_HOST_DEVICE constexpr int samples_per_16b(int kind) {
  return kind == kU4 ? 32 : 16 / elem_bytes(kind);
}
// Bytes of n raw samples (4-bit: rounded up to whole bytes).
DD_HOST_DEVICE constexpr int64_t sample_bytes(int kind, int64_t n) {
  return kind == kU4 ? (n + 1) / 2 : n * elem_bytes(kind);
}
// Decimated samples in 16 raw bytes: TMA copies start 16-byte aligned, so a
// window starts up to align_samples - 1 decimated samples before the block's
// base shift.  The tiled kernels take bins dividing the samples in 16 bytes.
DD_HOST_DEVICE constexpr int align_samples(int kind, int bin) {
  return samples_per_16b(kind) / bin;
}
// The bin the staged rows are at: packed copies are already decimated.
DD_HOST_DEVICE constexpr int staged_bin(int kind, int bin) {
  return packed_copy_kind(kind) ? 1 : bin;
}
inline bool bin_supported(int kind, int bin) {
  const int per = samples_per_16b(kind);
  return bin >= 1 && bin <= per && per % bin == 0 && (kind != kU8 || bin == 1) &&
         (!direct_kind(kind) || bin == 1) && (kind != kU4 || bin <= 16);
}
// Channels between widenings of the accumulators: uint8 pairs in 16-bit lanes
// hold 255 * 256 < 2^16 (packed copies of uint8 decimated by b: 65535 /
// (255 b) channels), 4-bit pairs 15 * bin per channel; one-sample words
// stay below 2^31 for floor((2^31 - 1) / (max sample * bin)) channels; float
// never needs one.
inline int flush_channels(int kind, int bin) {
  if (kind == kU8) return 256;
  if (kind == kU8P) return 65535 / (255 * bin);  // decimated uint8 sums (bin 1: 256)
  if (kind == kU4) return 65535 / (15 * bin);
  if (float_kind(kind)) return 1 << 30;
  const double max_sample = (kind == kU8W ? 255.0 : 65535.0) * bin;
  const double n = 2147483647.0 / max_sample;
  return n > (1 << 30) ? (1 << 30) : static_cast<int>(n);
}

// Tile shapes: DMs per lane (the register tile is dr DMs x kH words), warps
// per CTA, CTAs per SM and channels per pipeline stage.  Fewer DMs per lane
// free registers for more resident warps and admit steeper plans (a wider
// per-warp shift span) at the cost of more shared-memory traffic per add.
struct Shape {
  int dr;
  int warps;
  int min_blocks;
  int nc;
};
constexpr Shape kShapes[] = {{8, 8, 1, 16}, {6, 12, 1, 24}, {4, 12, 1, 24}, {2, 12, 1, 16},
                             {1, 12, 1, 16}};
// The persistent batch kernel serves these DMs-per-lane with one resource
// footprint (12 warps, one CTA per SM, 16 channels per stage); the DM blocks
// (records) only depend on DMs per lane and warps, so any 12-warp plan fits.
constexpr int kBatchWarps = 12;
constexpr int kBatchNc = 16;
constexpr int kBatchDr[] = {4, 2, 1};

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

// Pattern tiles (fwd_pattern.cu): every lane owns kPatDr consecutive DMs x H
// window words, H odd.  From one trial DM to the next the shift of channel c
// grows by the floor or the ceiling of step k_c / (bin t_samp) (Eq. 1 is
// linear in DM), so the increments i1, i2, i3 between a warp's four DMs are
// a or a + 1 for a = min(i1, i2, i3).  With a < kPatBases the offsets of the
// four DMs from the first, (0, i1, i1 + i2, i1 + i2 + i3), are one of
// kPatterns patterns, numbered 8 a + (i1 - a) + 2 (i2 - a) + 4 (i3 - a).
constexpr int kPatDr = 4;
constexpr int kPatBases = 4;
constexpr int kPatterns = 8 * kPatBases;
constexpr int kPatMaxWarps = 16;
constexpr int kPatOffBits = 11;      // window offset field of a pattern record entry
constexpr uint32_t kPatOffMask = (1u << kPatOffBits) - 1;

// Per (DM block of kPatDr * warps DMs, channel) record, 48 bytes.
struct PRec {
  int32_t base;                 // s(c, first DM of the block)
  int32_t pad[3];
  uint16_t w[kPatMaxWarps];     // warp w: window offset | pattern << kPatOffBits
};
static_assert(sizeof(PRec) == 48, "PRec must stay 48 bytes");

// Channel pairs: with `pairs`, each warp runs the channels of a stage as
// pairs that share its increment pattern, two samples per accumulator update
// (a three-input integer add), and the channels left without a partner one by
// one.  Per (DM block, stage) the host writes a chunk of per-warp lists: pair
// counts (kPairMaxWarps bytes), single counts (kPairMaxWarps bytes), then
// warps x nc items
// {a1 | a2 << 16, pattern}, pairs first, a = staged channel * lp + window
// offset.
constexpr int kPairMaxWarps = 32;
constexpr int kPairCountBytes = 2 * kPairMaxWarps;
struct PairItem {
  uint32_t a;    // a1 | a2 << 16 (word offsets into the window buffer)
  uint32_t pat;  // pattern number
};
static_assert(sizeof(PairItem) == 8, "PairItem must stay 8 bytes");

// Pattern tile shapes: window words per lane (odd), warps per CTA, channels
// per pipeline stage, channel pairs (integer kinds) or single channels (float
// kind), double-buffered window words (one barrier per stage), and the
// largest base increment a served.  Single-channel shapes with amax 1 load
// the lane's H + 6 window words before the pattern branch; the others load
// inside each pattern's block only the words its offsets touch.
struct PatShape {
  int h;
  int warps;
  int nc;
  bool pairs;
  bool dbuf;
  int amax;
};
// Fewer channels per stage fit the wider raw windows of larger bins.  Float:
// 32 channels per stage with loads inside the pattern blocks measured 12 %
// faster at H = 23 than H = 19 with loads before the branch (1024-channel
// float32 plan, 3.85 against 4.38 ms).
// Float pairs (kF32P, 64-bit words of two floats): H = 11 words of 2
// samples, the accumulators of 4 DMs in 88 registers (H = 13 with 12 warps),
// channel pairs (two add.f32x2 per accumulator) or single channels.
// The automatic choice takes the first entry that serves and fits; the
// entries from index kPatTuneFirst on are reached only through an explicit
// shape (dd_plan_set_tile_shape), for the autotuner: other window widths,
// warp counts and channels per stage.
// Float pairs take channel pairs first (two channels per indexed branch: the
// 1024-channel plan ran 2.94 ms against 3.07 ms with single channels).
constexpr PatShape kPatShapes[] = {
    {23, 16, 32, true, false, 3},  {23, 16, 12, true, false, 3},  {23, 16, 6, true, false, 3},
    {23, 16, 32, false, false, 3}, {19, 16, 32, false, false, 3}, {19, 16, 12, false, false, 1},
    {19, 16, 6, false, false, 1},  {19, 16, 12, false, false, 3}, {19, 16, 6, false, false, 3},
    {11, 16, 24, true, false, 3},  {11, 16, 16, true, false, 3},  {11, 16, 24, false, false, 3},
    {11, 16, 16, false, false, 3}, {11, 16, 8, false, false, 3},
    // Tuning entries.
    {21, 16, 32, true, false, 3},  {19, 16, 32, true, false, 3},  {25, 12, 32, true, false, 3},
    {23, 12, 32, true, false, 3},  {23, 16, 24, true, false, 3},  {21, 16, 32, false, false, 3},
    {13, 12, 16, false, false, 3}, {11, 12, 24, false, false, 3}, {13, 12, 16, true, false, 3},
    {11, 12, 24, true, false, 3}};
constexpr int kPatTuneFirst = 14;
constexpr int kNumPatShapes = static_cast<int>(sizeof(kPatShapes) / sizeof(kPatShapes[0]));
constexpr bool pat_shapes_fit_records() {
  for (const PatShape& s : kPatShapes)
    if (s.warps > (s.pairs ? kPairMaxWarps : kPatMaxWarps)) return false;
  return true;
}
static_assert(pat_shapes_fit_records(), "a pattern shape has more warps than its records hold");
// The shape serves a kind: float-pair shapes (H < 15) serve kF32P only, with
// channel pairs or single channels; the others pair integer window words or
// take float words one channel at a time.
DD_HOST_DEVICE constexpr bool pat_shape_serves(const PatShape& s, int kind) {
  return ((s.h < 15) == float_pairs(kind)) &&
         (s.pairs ? !float_kind(kind) || float_pairs(kind) : float_kind(kind)) &&
         (!direct_kind(kind) || !s.dbuf);
}

DD_HOST_DEVICE constexpr int pair_chunk_bytes(int warps, int nc) {
  return kPairCountBytes + warps * nc * static_cast<int>(sizeof(PairItem));
}

DD_HOST_DEVICE constexpr int pat_chunk_bytes(const PatShape& s) {
  return s.pairs ? pair_chunk_bytes(s.warps, s.nc) : 0;
}


constexpr size_t kRecOffset = 128;
DD_HOST_DEVICE constexpr size_t raw_offset(int nc, int rec_bytes = static_cast<int>(sizeof(Rec))) {
  return (kRecOffset + 2 * static_cast<size_t>(nc) * rec_bytes + 127) / 128 * 128;
}

// Words of a channel's staged window for a given DM-block shift span.
inline int32_t window_words(int kind, int bin, int32_t span) {
  const int32_t need = kH * 31 + span + (align_samples(kind, bin) - 1) + kWin;
  return (need + 15) / 16 * 16;
}

// Raw bytes fetched per channel and stage for lp window words (uint8 at bin 1
// also fetches the paired samples, `pair` words further).
DD_HOST_DEVICE constexpr int32_t raw_bytes(int kind, int bin, int32_t lp, int pair = kPair) {
  return kind == kU8   ? lp + pair
         : kind == kU4 ? (lp + pair) * bin / 2
                       : lp * elem_bytes(kind) * bin;
}

// Pattern tiles: output samples per CTA tile, staged window words per channel
// for a DM-block shift span, and shared memory.
DD_HOST_DEVICE constexpr int pat_tile_samples(int kind, int h) {
  return 32 * h * samples_per_word(kind);
}
inline int32_t pat_window_words(int kind, int bin, int h, int32_t span) {
  // A lane reads at most h + 6 words from its first DM's offset (the loads
  // before the branch) or, inside a pattern block, up to its last DM's shift
  // plus h: lane 31 stays below 31h + (span + align - 1) + h + 6.
  const int32_t need = 32 * h + span + (align_samples(kind, bin) - 1) + 6;
  // Whole 16-byte raw windows: 4-bit pairs need lp + 32h to be even in 16s.
  const int32_t mult = kind == kU4 ? 32 : 16;
  return (need + mult - 1) / mult * mult;
}
// Pattern tiles' shared memory: 128 bytes of barriers, two record buffers
// (PRec per channel, or one pair chunk per stage), one raw buffer of nc
// channels, and one window buffer (two with dbuf).
DD_HOST_DEVICE constexpr size_t pat_raw_offset(const PatShape& s) {
  return (kRecOffset +
          2 * static_cast<size_t>(s.pairs ? pat_chunk_bytes(s)
                                          : s.nc * static_cast<int>(sizeof(PRec))) +
          127) / 128 * 128;
}
// Raw bytes staged per channel.
DD_HOST_DEVICE constexpr int32_t pat_raw_bytes(int kind, int bin, const PatShape& s, int32_t lp) {
  return raw_bytes(kind, bin, lp, 32 * s.h);
}
// Direct kinds stage window words: two staging buffers and no window buffer.
inline size_t pat_smem_bytes(int kind, int bin, const PatShape& s, int32_t lp) {
  if (direct_kind(kind))
    return pat_raw_offset(s) + 2 * static_cast<size_t>(s.nc) * pat_raw_bytes(kind, bin, s, lp);
  return pat_raw_offset(s) + static_cast<size_t>(s.nc) * pat_raw_bytes(kind, bin, s, lp) +
         (s.dbuf ? 2 : 1) * static_cast<size_t>(s.nc) * lp * 4;
}

inline size_t smem_bytes(int kind, int bin, const Shape& s, int32_t lp) {
  return raw_offset(s.nc) + 2 * static_cast<size_t>(s.nc) * raw_bytes(kind, bin, lp) +
         static_cast<size_t>(s.nc) * lp * 4;
}

// One (DM block, time tile) work unit of one range.
struct TileParams {
  const void* x;        // channel-major input rows
  int64_t stride;       // elements between channel rows (and the rows' length)
  int64_t x_origin;     // staged sample held by element 0 of each row (0, or a
                        // time segment's first word in a ring slot)
  int32_t align;        // window starts: multiples of this many staged samples
  int32_t n_chan;
  const void* recs;     // [n_blocks][n_chan] Rec or PRec; pair chunks [n_blocks][stages]
  const int32_t* bases; // pair tiles: s(c, first DM of block) [n_blocks][n_chan]
  int32_t chunk_bytes;  // pair tiles: bytes per (DM block, stage) chunk
  int32_t n_dm;
  int32_t n_blocks;
  int64_t n_out;        // output row length
  int64_t out_stride;   // elements from output row d to row d + 1 (n_out, or negative)
  int64_t tile0;        // first time tile of the launch
  int64_t t_end;        // outputs t >= t_end are not written (<= n_out)
  int32_t lp;           // window words per staged channel
  int32_t lraw;         // raw bytes per staged channel
  uint32_t units_magic; // u / (lp/4) == (u * magic) >> (32 + shift)
  int32_t units_shift;
  int32_t bin;          // time decimation of the range (raw samples per window word)
  int32_t flush;        // channels between accumulator widenings
  void* out;            // [n_dm][n_out] int32 or float32
  int32_t* err;
  int32_t wait_iters;   // polls before a pipeline wait gives up (kWaitIters by default)
  int32_t hold_stage;   // channel stage whose copies are never issued (timeout test; -1: none)
  // Widening slots of the pattern tiles with 16-bit lanes (nullptr: widen
  // into the output rows).  A CTA holds one slot for the duration of a unit:
  // each warp widens its lanes into its own part of the slot (64-bit words
  // of the sums for samples u and u + 32 H) whenever its lanes are full, and
  // the unit's last stage adds the slot to the lanes and stores each output
  // once (the slots of the CTAs in flight, 57 MB at paper scale, stay in L2).  The slots live in the plan workspace; wflags[s] is 1 while slot s
  // is held.
  unsigned long long* wslots;
  int32_t* wflags;
  int32_t n_wslots;
  int32_t wslot_words;  // 64-bit words per slot
};
// Widening mode of a pattern-tile launch (a template argument of its
// kernel): 0 into the output rows, 1 into slots (every word when the lanes
// are full), G = 8 (and for packed copies of binned uint8, G = 4 or 2) into
// slots by G phases: the lanes take exactly G stages of nc channels, and 1 / G
// of the words widen after every stage.  Separate kernels: one that could
// take either of 0 and 1 at run time was 3 % slower on the paper plan.
DD_HOST_DEVICE constexpr int widen_mode(int kind, int nc, bool slots, int32_t flush) {
  return !packed_pairs(kind) || !slots                      ? 0
         : flush / nc == 8                                  ? 8
         : kind == kU8P && (flush / nc == 4 || flush / nc == 2) ? flush / nc
                                                                : 1;
}
// Widening slots in a plan workspace: two per SM of the largest GB300-class
// part.  Every kernel that takes slots holds at most one CTA per SM (16 warps
// at 128 registers per thread, or 12 warps at up to 168, fill the register
// file), so the CTAs of all launches of a plan in flight at once, on any
// streams, find a free slot; the second half is margin.
constexpr int kWidenSlots = 320;

// Persistent batch execution: one work list of (job, DM block, time tile)
// items over many jobs (plan ranges with their input/output pointers).
struct BatchJob {
  TileParams p;
  int32_t kind;  // kU8 / kU8W / kU16 / kF32
  int32_t dr;    // DMs per lane (a kBatchShapes entry)
};

struct BatchItem {
  int32_t job;
  int32_t blk;
  int32_t tile;
  int32_t pad;
};

struct BatchArgs {
  const BatchJob* jobs;    // device
  const BatchItem* items;  // device, in execution order
  int32_t n_items;
  uint32_t* counter;       // device, zero before the launch
  int32_t max_lraw;        // largest raw window of any job (shared-memory layout)
};

// Persistent batch execution of pattern-tile jobs (fwd_pattern_batch.cu):
// every job names its kind and its tk::kPatShapes entry.
struct PatBatchJob {
  TileParams p;
  int32_t kind;
  int32_t shape;
};

struct PatBatchArgs {
  const PatBatchJob* jobs;  // device
  const BatchItem* items;   // device, in execution order
  int32_t n_items;
  uint32_t* counter;        // device, zero before the launch
};

inline size_t batch_smem_bytes(int32_t max_lraw, int32_t max_lp) {
  return raw_offset(kBatchNc) + 2 * static_cast<size_t>(kBatchNc) * max_lraw +
         static_cast<size_t>(kBatchNc) * max_lp * 4;
}

}  // namespace tk
}  // namespace dd
