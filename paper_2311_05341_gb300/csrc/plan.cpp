// plan.cpp -- host planner: per-channel delay coefficients and integer shift
// tables in FP64, DM blocking and the device workspace layout.
//
// The shift of channel c at trial DM_d of a range with time bin b is
//   s(c, d) = floor(DM_d * k_c / (b * t_samp) + 0.5),
//   k_c     = C_DM * (1/f_c^2 - 1/f_ref^2)              (Eq. 1, Eq. 7 form),
//   DM_d    = lo + d * step                             (fixed step, Table 2),
// evaluated in exactly this order in FP64.  This file is compiled with
// -ffp-contract=off so no multiply-add is fused: the table must not depend on
// the host CPU.  The kernels never evaluate the delay law; they read the
// precomputed integer shifts, like the paper's precomputed Delta t_pc array
// (Sec. 4.1) but resolved to integers on the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <iterator>
#include <map>
#include <utility>
#include <vector>

#include "dd_internal.h"
#include "fwd_tiled.h"

namespace dd {

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Delay of one (channel, DM) in decimated samples, before rounding.
double delay_samples(double dm, double k_c, int32_t bin, double t_samp) {
  double delay = dm * k_c;
  double tick = static_cast<double>(bin) * t_samp;
  return delay / tick;
}

// Max over DM blocks of `per_block` DMs and over channels of the in-block span
// s(c, last DM of block) - s(c, first DM of block).
int32_t block_span(const RangePlan& rp, int32_t n_chan, int32_t per_block) {
  int32_t span = 0;
  for (int64_t d0 = 0; d0 < rp.n_dm; d0 += per_block) {
    int64_t d1 = std::min<int64_t>(d0 + per_block, rp.n_dm) - 1;
    const int32_t* a = &rp.shifts[static_cast<size_t>(d0) * n_chan];
    const int32_t* b = &rp.shifts[static_cast<size_t>(d1) * n_chan];
    for (int32_t c = 0; c < n_chan; ++c) span = std::max(span, b[c] - a[c]);
  }
  return span;
}

// Records of the register-tiled kernel for a tile shape with dr DMs per lane
// and W warps.  For DM block b (first DM d0, dr * W DMs), channel c and warp w
// (DMs d0 + dr*w + i, i < dr, clamped to the last DM):
//   base  = s(c, d0),  m = base mod A (A samples in 16 bytes: the TMA copy of
//           the channel's window starts 16-byte aligned),
//   D_i   = s(c, d0 + dr*w + i) - base + m   (word offset inside the staged window),
//   a_w   = 4 * floor(D_0 / 4)                (16-byte aligned window start),
//   off_i = D_i - a_w                          (must fit in 4 bits).
// Returns false if some offset does not fit.
bool build_tile_records(const RangePlan& rp, int32_t n_chan, int kind, const tk::Shape& sh,
                        std::vector<tk::Rec>& recs, int32_t* n_blocks_out) {
  using namespace tk;
  const int dm_cta = sh.dr * sh.warps;
  const int32_t align = align_samples(kind, tk::staged_bin(kind, rp.r.bin));
  const int64_t n_blocks = (rp.n_dm + dm_cta - 1) / dm_cta;
  recs.assign(static_cast<size_t>(n_blocks) * n_chan, tk::Rec{});
  for (int64_t b = 0; b < n_blocks; ++b) {
    const int64_t d0 = b * dm_cta;
    for (int32_t c = 0; c < n_chan; ++c) {
      tk::Rec& r = recs[static_cast<size_t>(b) * n_chan + c];
      const int32_t base = rp.shifts[static_cast<size_t>(d0) * n_chan + c];
      const int32_t m = base % align;
      r.base = base;
      for (int w = 0; w < sh.warps; ++w) {
        int32_t a_w = 0;
        uint32_t packed = 0;
        for (int i = 0; i < sh.dr; ++i) {
          const int64_t d = std::min<int64_t>(d0 + w * sh.dr + i, rp.n_dm - 1);
          const int32_t D = rp.shifts[static_cast<size_t>(d) * n_chan + c] - base + m;
          if (i == 0) a_w = (D >> 2) << 2;
          const int32_t off = D - a_w;
          if (off < 0 || off > kMaxOff) return false;
          packed |= static_cast<uint32_t>(off) << (4 * i);
        }
        if ((a_w >> 2) > 255) return false;
        r.delta[w] = packed;
        r.aq[w] = static_cast<uint8_t>(a_w >> 2);
      }
    }
  }
  *n_blocks_out = static_cast<int32_t>(n_blocks);
  return true;
}

// Pattern number of the increments i_k = s(c, d_k) - s(c, d_{k-1}) (k = 1..3)
// of a warp's DMs d_0..d_3, of which the first n_real are trial DMs of the
// range: 8 a + sum_k (i_k - a) 2^(k-1), a = min_k i_k.  False unless every
// i_k is a or a + 1 and 0 <= a <= amax.  DMs past the end of the range are
// never stored: they take increment a (at most 6 samples past the last DM,
// inside the window's slack).
bool pattern_of(const int32_t* s_dm, int n_real, int amax, uint32_t* pat) {
  using tk::kPatDr;
  *pat = 0;
  if (n_real <= 1) return true;
  int32_t inc[kPatDr - 1];
  int32_t a = s_dm[1] - s_dm[0];
  for (int k = 1; k < n_real; ++k) {
    inc[k - 1] = s_dm[k] - s_dm[k - 1];
    a = std::min(a, inc[k - 1]);
  }
  if (a < 0 || a > amax) return false;
  uint32_t bits = 0;
  for (int k = 0; k + 1 < n_real; ++k) {
    if (inc[k] - a > 1) return false;
    bits |= static_cast<uint32_t>(inc[k] - a) << k;
  }
  *pat = 8u * static_cast<uint32_t>(a) + bits;
  return true;
}

// Records of the pattern kernel for shape ps (kPatDr DMs per lane, ps.warps
// warps).  For DM block b (first DM d0), channel c and warp w (DMs
// d_i = d0 + kPatDr w + i, clamped to the last DM):
//   base = s(c, d0),  m = base mod A (as for the offset tiles),
//   off  = s(c, d_0) - base + m     (window offset, kPatOffBits bits),
//   entry = off | pattern_of(s(c, d_0..d_3)) << kPatOffBits.
// Returns false if some offset or increment does not fit.
bool build_pattern_records(const RangePlan& rp, int32_t n_chan, int kind, const tk::PatShape& ps,
                           std::vector<tk::PRec>& recs, int32_t* n_blocks_out) {
  using namespace tk;
  const int dm_cta = kPatDr * ps.warps;
  const int32_t align = align_samples(kind, tk::staged_bin(kind, rp.r.bin));
  const int64_t n_blocks = (rp.n_dm + dm_cta - 1) / dm_cta;
  recs.assign(static_cast<size_t>(n_blocks) * n_chan, tk::PRec{});
  auto shift = [&](int64_t d, int32_t c) {
    d = std::min<int64_t>(d, rp.n_dm - 1);
    return rp.shifts[static_cast<size_t>(d) * n_chan + c];
  };
  for (int64_t b = 0; b < n_blocks; ++b) {
    const int64_t d0 = b * dm_cta;
    for (int32_t c = 0; c < n_chan; ++c) {
      tk::PRec& r = recs[static_cast<size_t>(b) * n_chan + c];
      const int32_t base = shift(d0, c);
      const int32_t m = base % align;
      r.base = base;
      for (int w = 0; w < ps.warps; ++w) {
        const int64_t dw = d0 + static_cast<int64_t>(kPatDr) * w;
        const int32_t off = shift(dw, c) - base + m;
        if (off < 0 || off > static_cast<int32_t>(kPatOffMask)) return false;
        int32_t s_dm[kPatDr];
        for (int i = 0; i < kPatDr; ++i) s_dm[i] = shift(dw + i, c);
        const int n_real = static_cast<int>(std::min<int64_t>(kPatDr, rp.n_dm - dw));
        uint32_t pat = 0;
        if (!pattern_of(s_dm, n_real, ps.amax, &pat)) return false;
        r.w[w] = static_cast<uint16_t>(static_cast<uint32_t>(off) | pat << kPatOffBits);
      }
    }
  }
  *n_blocks_out = static_cast<int32_t>(n_blocks);
  return true;
}

// Channel-pair tables of the pattern kernel for shape ps (ps.pairs): the base
// shifts s(c, d0) of every (DM block, channel) as int32, padded to 256 bytes,
// then one chunk per (DM block, stage of ps.nc channels).  In a chunk, warp w
// lists the stage's channels as pairs of equal pattern (entries as in
// build_pattern_records), grouped by pattern, then the channels left alone.
// Item word offsets a = staged channel * lp + off must stay below 2^16.  Returns false if some offset or increment does not fit.
bool build_pair_tables(const RangePlan& rp, int32_t n_chan, int kind, const tk::PatShape& ps,
                       int32_t lp, std::vector<unsigned char>& out, size_t* chunk_off,
                       int32_t* n_blocks_out) {
  using namespace tk;
  const int dm_cta = kPatDr * ps.warps;
  const int32_t align = align_samples(kind, tk::staged_bin(kind, rp.r.bin));
  const int64_t n_blocks = (rp.n_dm + dm_cta - 1) / dm_cta;
  const int n_st = (n_chan + ps.nc - 1) / ps.nc;
  const size_t cb = static_cast<size_t>(pair_chunk_bytes(ps.warps, ps.nc));
  const size_t bases_bytes = align_up(static_cast<size_t>(n_blocks) * n_chan * 4, 256);
  out.assign(bases_bytes + static_cast<size_t>(n_blocks) * n_st * cb, 0);
  auto shift = [&](int64_t d, int32_t c) {
    d = std::min<int64_t>(d, rp.n_dm - 1);
    return rp.shifts[static_cast<size_t>(d) * n_chan + c];
  };
  std::vector<std::vector<uint32_t>> by_pat(kPatterns);
  for (int64_t b = 0; b < n_blocks; ++b) {
    const int64_t d0 = b * dm_cta;
    int32_t* bases = reinterpret_cast<int32_t*>(out.data()) + b * n_chan;
    for (int32_t c = 0; c < n_chan; ++c) bases[c] = shift(d0, c);
    for (int st = 0; st < n_st; ++st) {
      unsigned char* chunk = out.data() + bases_bytes + (static_cast<size_t>(b) * n_st + st) * cb;
      PairItem* items = reinterpret_cast<PairItem*>(chunk + kPairCountBytes);
      const int c0 = st * ps.nc, nc = std::min(ps.nc, n_chan - c0);
      for (int w = 0; w < ps.warps; ++w) {
        for (auto& v : by_pat) v.clear();
        const int64_t dw = d0 + static_cast<int64_t>(kPatDr) * w;
        for (int k = 0; k < nc; ++k) {
          const int32_t c = c0 + k;
          const int32_t base = bases[c];
          const int32_t off = shift(dw, c) - base + base % align;
          if (off < 0 || off > static_cast<int32_t>(kPatOffMask)) return false;
          int32_t s_dm[kPatDr];
          for (int i = 0; i < kPatDr; ++i) s_dm[i] = shift(dw + i, c);
          const int n_real = static_cast<int>(std::min<int64_t>(kPatDr, rp.n_dm - dw));
          uint32_t pat = 0;
          if (!pattern_of(s_dm, n_real, ps.amax, &pat)) return false;
          const uint32_t a = static_cast<uint32_t>(k) * lp + static_cast<uint32_t>(off);
          if (a > 0xffffu) return false;
          by_pat[pat].push_back(a);
        }
        int n = 0;
        for (uint32_t pat = 0; pat < static_cast<uint32_t>(kPatterns); ++pat) {
          const auto& v = by_pat[pat];
          for (size_t i = 0; i + 1 < v.size(); i += 2)
            items[w * ps.nc + n++] = PairItem{v[i] | v[i + 1] << 16, pat};
        }
        chunk[w] = static_cast<unsigned char>(n);
        const int n_pairs = n;
        for (uint32_t pat = 0; pat < static_cast<uint32_t>(kPatterns); ++pat)
          if (by_pat[pat].size() % 2) items[w * ps.nc + n++] = PairItem{by_pat[pat].back(), pat};
        chunk[kPairMaxWarps + w] = static_cast<unsigned char>(n - n_pairs);
      }
    }
  }
  *chunk_off = bases_bytes;
  *n_blocks_out = static_cast<int32_t>(n_blocks);
  return true;
}

// Multiply-high constants for exact u / d with u < limit (verified exhaustively).
bool division_magic(uint32_t d, uint32_t limit, uint32_t* magic, int32_t* shift) {
  int32_t s = 0;
  while ((2u << s) <= d) ++s;  // s = floor(log2(d))
  // One lower first: a power of two d = 2^s needs m = 2^31 at shift s - 1
  // (2^32 at shift s does not fit 32 bits).  Every candidate is verified.
  if (s > 0) --s;
  for (; s < 32; ++s) {
    const uint64_t m = ((uint64_t{1} << (32 + s)) + d - 1) / d;
    if (m > 0xffffffffull) break;
    bool ok = true;
    for (uint32_t u = 0; u < limit && ok; ++u)
      ok = ((static_cast<uint64_t>(u) * m) >> (32 + s)) == u / d;
    if (ok) {
      *magic = static_cast<uint32_t>(m);
      *shift = s;
      return true;
    }
  }
  return false;
}


// Try one tile shape for a range; on success fill the range's tile fields.
bool try_tile_shape(RangePlan& rp, int32_t n_chan, int kind, const tk::Shape& sh) {
  // 4-bit input and the direct kinds run on the pattern tiles only.
  if (kind == tk::kU4 || tk::direct_kind(kind)) return false;
  const int32_t span = block_span(rp, n_chan, sh.dr * sh.warps);
  const int32_t lp = tk::window_words(kind, rp.r.bin, span);
  if (tk::smem_bytes(kind, rp.r.bin, sh, lp) > 227 * 1024) return false;  // one CTA per SM at worst
  uint32_t magic = 0;
  int32_t shift = 0;
  if (!division_magic(static_cast<uint32_t>(lp / 4), static_cast<uint32_t>(sh.nc * lp / 4), &magic,
                      &shift))
    return false;
  std::vector<tk::Rec> recs;
  int32_t n_blocks = 0;
  if (!build_tile_records(rp, n_chan, kind, sh, recs, &n_blocks)) return false;
  rp.tile_ok = true;
  rp.tile_pattern = false;
  rp.tile_dr = sh.dr;
  rp.tile_h = tk::kH;
  rp.tile_shape = 0;
  rp.tile_chunk_off = 0;
  rp.tile_chunk_bytes = 0;
  rp.tile_kind = kind;
  rp.tile_n_blocks = n_blocks;
  rp.tile_lp = lp;
  rp.tile_units_magic = magic;
  rp.tile_units_shift = shift;
  rp.tile_recs.resize(recs.size() * sizeof(tk::Rec));
  std::memcpy(rp.tile_recs.data(), recs.data(), rp.tile_recs.size());
  return true;
}

// Try one pattern shape (index `shape` of tk::kPatShapes).
bool try_pattern_shape(RangePlan& rp, int32_t n_chan, int kind, int shape) {
  const tk::PatShape& ps = tk::kPatShapes[shape];
  if (!tk::pat_shape_serves(ps, kind)) return false;
  const int32_t span = block_span(rp, n_chan, tk::kPatDr * ps.warps);
  const int sb = tk::staged_bin(kind, rp.r.bin);
  const int32_t lp = tk::pat_window_words(kind, sb, ps.h, span);
  if (tk::pat_smem_bytes(kind, sb, ps, lp) > 227 * 1024) return false;
  uint32_t magic = 0;
  int32_t shift = 0;
  if (!division_magic(static_cast<uint32_t>(lp / 4), static_cast<uint32_t>(ps.nc * lp / 4),
                      &magic, &shift))
    return false;
  std::vector<unsigned char> tables;
  int32_t n_blocks = 0;
  size_t chunk_off = 0;
  if (ps.pairs) {
    if (!build_pair_tables(rp, n_chan, kind, ps, lp, tables, &chunk_off, &n_blocks)) return false;
  } else {
    std::vector<tk::PRec> recs;
    if (!build_pattern_records(rp, n_chan, kind, ps, recs, &n_blocks)) return false;
    tables.resize(recs.size() * sizeof(tk::PRec));
    std::memcpy(tables.data(), recs.data(), tables.size());
  }
  rp.tile_ok = true;
  rp.tile_pattern = true;
  rp.tile_dr = tk::kPatDr;
  rp.tile_h = ps.h;
  rp.tile_shape = shape;
  rp.tile_kind = kind;
  rp.tile_n_blocks = n_blocks;
  rp.tile_lp = lp;
  rp.tile_units_magic = magic;
  rp.tile_units_shift = shift;
  rp.tile_chunk_off = chunk_off;
  rp.tile_chunk_bytes = tk::pat_chunk_bytes(ps);
  rp.tile_recs = std::move(tables);
  return true;
}

// Register-tiled kernel: a supported time bin (bin * sample bytes divides 16)
// and a tile shape whose per-warp DM offsets fit the 4-bit fields and whose
// window fits shared memory.  uint8 at bin 1 packs two samples per word; at a
// larger bin it keeps one decimated sample per word.  The automatic choice
// takes the pattern tile when every per-DM shift increment is 0, 1 or 2 (it
// ran 1.2x to 1.8x faster than the best offset tile on every plan measured),
// else the first offset shape that fits in kAutoOrder (fewer DMs per lane
// serve steeper plans; 8 DMs per lane stages 16 channels, fitting the widest
// raw windows of large bins).
void choose_tile(RangePlan& rp, int32_t n_chan, dd_dtype dtype) {
  static const int kAutoOrder[] = {6, 4, 2, 1, 8};
  rp.tile_ok = false;
  rp.tile_pattern = false;
  rp.tile_dr = 0;
  rp.tile_h = 0;
  rp.tile_kind = 0;
  rp.tile_chunk_off = 0;
  rp.tile_chunk_bytes = 0;
  rp.alt_kind = 0;
  rp.tile_recs.clear();
  // Packed input at bin 1: uint8 and 4-bit share the paired word format,
  // uint16 is widened to one sample per word.
  // Packed copies: uint8, 4-bit, uint16 and float32 at bin 1; uint8 also
  // decimated by 2, 4 or 8 (sums of at most 2040 keep 32 or more channels in
  // a 16-bit lane).
  const int b = rp.r.bin;
  const bool packed = rp.tile_request == DD_TILE_PACKED &&
                      (dtype == DD_U8 || dtype == DD_U4 || dtype == DD_U16 || dtype == DD_F32) &&
                      (b == 1 || (dtype == DD_U8 && (b == 2 || b == 4 || b == 8)));
  const int kind = packed ? (dtype == DD_U16   ? tk::kU16P
                             : dtype == DD_F32 ? tk::kF32P
                                               : tk::kU8P)
                   : dtype == DD_U4                   ? tk::kU4
                   : (dtype == DD_U8 && rp.r.bin > 1) ? tk::kU8W
                                                      : static_cast<int>(dtype);
  if (rp.tile_request == DD_TILE_PACKED && !tk::packed_copy_kind(kind)) return;
  if (!tk::bin_supported(kind, tk::staged_bin(kind, rp.r.bin))) return;
  if (rp.tile_request == DD_TILE_PATTERN || rp.tile_request == DD_TILE_PACKED ||
      rp.tile_request == 0) {
    // Float32 at bin 1 first tries the direct kind (the input words are the
    // window words: no unpacking, two staging buffers).  An explicit shape
    // (the autotuner's) is the only one tried; otherwise the first entry
    // before the tuning entries that serves and fits.
    auto candidate = [&](int i) {
      return rp.shape_request >= 0 ? i == rp.shape_request : i < tk::kPatTuneFirst;
    };
    if (kind == tk::kF32 && rp.r.bin == 1)
      for (int i = 0; i < tk::kNumPatShapes; ++i)
        if (candidate(i) && try_pattern_shape(rp, n_chan, tk::kF32D, i)) return;
    for (int i = 0; i < tk::kNumPatShapes; ++i)
      if (candidate(i) && try_pattern_shape(rp, n_chan, kind, i)) {
        // The automatic tile of uint8, 4-bit or uint16 input at bin 1 can
        // also run from a packed copy (dd_run_scratch with the scratch of
        // dd_plan_packed_scratch_bytes): same tables, the packed kernel's
        // two staging buffers must fit shared memory too.
        const int alt = kind == tk::kU16 ? static_cast<int>(tk::kU16P)
                                         : static_cast<int>(tk::kU8P);
        const tk::PatShape& ps = tk::kPatShapes[i];
        if (rp.tile_request == 0 && rp.shape_request < 0 && b == 1 &&
            (kind == tk::kU8 || kind == tk::kU4 || kind == tk::kU16) &&
            tk::pat_shape_serves(ps, alt) &&
            tk::pat_smem_bytes(alt, 1, ps, rp.tile_lp) <= 227 * 1024)
          rp.alt_kind = alt;
        return;
      }
    if (rp.tile_request != 0) return;
  }
  if (rp.tile_request > 0) {
    const tk::Shape* sh = tk::shape_for(rp.tile_request);
    if (sh) try_tile_shape(rp, n_chan, kind, *sh);
    return;
  }
  for (int dr : kAutoOrder)
    if (try_tile_shape(rp, n_chan, kind, *tk::shape_for(dr))) return;
}

// The adjoint of range rp (float32) as a forward transform: with P = s_max,
// xbar_r[c][u] = sum_d ybar[d][u - s(c, d)] = sum_d Z[d][u + P - s(c, d)] for
// the cotangent rows Z[d] padded with P zeros on both sides, so it is Eq. 3 on
// "channels" d (the range's trial DMs) at "trial DMs" c' = n_chan - 1 - c
// (the channels in reverse order) with shifts P - s(c, d) >= 0.  Those grow
// with c' by the delay differences of adjacent channels (small and
// non-negative for channels ordered from high to low frequency), which the
// pattern tiles serve when each warp's increments are a or a + 1.
void build_adjoint_range(const RangePlan& rp, int32_t n_chan, RangePlan* ar) {
  *ar = RangePlan{};
  ar->r = rp.r;
  ar->r.bin = 1;  // the cotangent rows are already at the range's time resolution
  ar->n_dm = n_chan;
  ar->tile_n_chan = static_cast<int32_t>(rp.n_dm);
  const int32_t pad = rp.s_max;
  const int64_t n_dm = rp.n_dm;
  ar->shifts.resize(static_cast<size_t>(n_chan) * n_dm);
  int32_t smax = 0;
  for (int32_t cp = 0; cp < n_chan; ++cp) {
    const int32_t c = n_chan - 1 - cp;
    for (int64_t d = 0; d < n_dm; ++d) {
      const int32_t sh = pad - rp.shifts[static_cast<size_t>(d) * n_chan + c];
      ar->shifts[static_cast<size_t>(cp) * n_dm + d] = sh;
      smax = std::max(smax, sh);
    }
  }
  ar->s_max = smax;
  if (n_dm > (int64_t{1} << 20)) return;
  // Float pairs first (two adds per instruction; the adjoint packs its padded
  // cotangent rows into pairs anyway), then plain floats.
  for (int kind : {static_cast<int>(tk::kF32P), static_cast<int>(tk::kF32D),
                   static_cast<int>(tk::kF32)})
    for (int i = 0; i < tk::kNumPatShapes; ++i)
      if (try_pattern_shape(*ar, static_cast<int32_t>(n_dm), kind, i)) return;
}

void layout_workspace(dd_plan_s* p) {
  size_t ws = tk::kStatusBytes;  // device status word(s) first
  auto place = [&](RangePlan& rp) {
    ws = align_up(ws, 256);
    rp.off_shifts = ws;
    ws += rp.shifts.size() * sizeof(int32_t);
    if (rp.tile_ok) {
      ws = align_up(ws, 256);
      rp.off_tile_recs = ws;
      ws += rp.tile_recs.size();
    }
  };
  for (auto& rp : p->ranges) place(rp);
  for (auto& ar : p->adj) place(ar);
  // Widening slots for the pattern tiles whose lanes hold 16-bit sums (uint8
  // and 4-bit, from the input or a packed copy): flags (zero: free) in the
  // uploaded image, the slots after it.
  p->wslot_words = 0;
  for (const auto& rp : p->ranges)
    if (rp.tile_ok && rp.tile_pattern && tk::packed_pairs(rp.tile_kind))
      p->wslot_words = std::max<int32_t>(
          p->wslot_words, tk::kPatDr * tk::kPatShapes[rp.tile_shape].warps * 32 * rp.tile_h);
  size_t image = align_up(ws, 256);
  if (p->wslot_words > 0) {
    p->off_wflags = image;
    image = align_up(image + tk::kWidenSlots * sizeof(int32_t), 256);
    p->off_wslots = image;
    p->ws_bytes = image + static_cast<size_t>(tk::kWidenSlots) * p->wslot_words * 8;
  } else {
    p->off_wflags = p->off_wslots = 0;
    p->ws_bytes = image;
  }
  p->host_ws.assign(image, 0);
  auto copy = [&](const RangePlan& rp) {
    std::memcpy(p->host_ws.data() + rp.off_shifts, rp.shifts.data(),
                rp.shifts.size() * sizeof(int32_t));
    if (rp.tile_ok)
      std::memcpy(p->host_ws.data() + rp.off_tile_recs, rp.tile_recs.data(), rp.tile_recs.size());
  };
  for (const auto& rp : p->ranges) copy(rp);
  for (const auto& ar : p->adj) copy(ar);
}

}  // namespace

int32_t dm_plan_ranges(const double* freqs, int32_t n_chan, double t_samp, double dm_max,
                       double tol, double width, int32_t max_bin, int32_t max_ranges,
                       dd_range* out) {
  double f_lo = freqs[0], f_hi = freqs[0];
  for (int32_t c = 1; c < n_chan; ++c) {
    f_lo = std::min(f_lo, freqs[c]);
    f_hi = std::max(f_hi, freqs[c]);
  }
  const double df = (f_hi - f_lo) / (n_chan - 1);
  const double f_c = 0.5 * (f_lo + f_hi);
  const double chan_per_dm = 8297.4e3 * df / (f_c * f_c * f_c) * 1e-3;  // s per unit DM (Eq. 4)
  const double k_band = kDispersionConstant * (1.0 / (f_lo * f_lo) - 1.0 / (f_hi * f_hi));
  const double q = 2.0 * std::sqrt(tol * tol - 1.0) / k_band;
  auto width_at = [&](double dm, int32_t b) {
    const double ts = b * t_samp, tc = chan_per_dm * dm;
    return std::sqrt(ts * ts + tc * tc + width * width);
  };
  int32_t n = 0;
  double lo = 0.0;
  int32_t bin = 1;
  while (lo < dm_max && n < max_ranges) {
    const double w0 = width_at(lo, bin);
    const double step = q * w0;
    double hi = dm_max;
    if (n + 1 < max_ranges) {
      // Where the continuous step has doubled: W_b(DM) = 2 W_b(lo).
      const double rest = 4.0 * w0 * w0 - (bin * t_samp) * (bin * t_samp) - width * width;
      if (chan_per_dm > 0.0) hi = std::min(hi, std::sqrt(std::max(rest, 0.0)) / chan_per_dm);
      // Where binning by 2 b costs little: t_chan = 2 b t_samp.
      if (2 * bin <= max_bin && chan_per_dm > 0.0)
        hi = std::min(hi, 2.0 * bin * t_samp / chan_per_dm);
    }
    // Trials lo + k step, k < n; the next range's first trial is hi.  The last
    // range keeps dm_max within half a step of its last trial.
    const bool last = hi >= dm_max;
    const double n_steps =
        std::max(1.0, std::ceil((hi - lo) / step + (last ? 0.5 : 0.0) - 1e-9));
    hi = lo + n_steps * step;
    out[n++] = dd_range{lo, hi, step, bin};
    if (2 * bin <= max_bin && chan_per_dm * hi >= 2.0 * bin * t_samp) bin *= 2;
    lo = hi;
  }
  return n;
}

int64_t range_n_out(const dd_plan_s* p, const RangePlan& rp, int64_t n_samp) {
  (void)p;
  return n_samp / rp.r.bin - rp.s_max;
}

dd_status build_plan(dd_plan_s* p) {
  const int32_t n_chan = p->n_chan;
  p->k.resize(n_chan);
  const double inv_ref2 = 1.0 / (p->f_ref * p->f_ref);
  for (int32_t c = 0; c < n_chan; ++c) {
    double f = p->freqs[c];
    double inv_f2 = 1.0 / (f * f);
    p->k[c] = kDispersionConstant * (inv_f2 - inv_ref2);
  }

  for (auto& rp : p->ranges) {
    rp.n_dm = std::llround((rp.r.dm_hi - rp.r.dm_lo) / rp.r.dm_step);
    if (rp.n_dm <= 0 || rp.n_dm > (int64_t{1} << 24))
      return fail(DD_ERR_INVALID_ARG, "range has no trial DMs or too many (max 2^24)");
    rp.shifts.resize(static_cast<size_t>(rp.n_dm) * n_chan);
    int32_t smax = 0;
    for (int64_t d = 0; d < rp.n_dm; ++d) {
      double dm = rp.r.dm_lo + static_cast<double>(d) * rp.r.dm_step;
      int32_t* row = &rp.shifts[static_cast<size_t>(d) * n_chan];
      for (int32_t c = 0; c < n_chan; ++c) {
        double x = delay_samples(dm, p->k[c], rp.r.bin, p->t_samp);
        if (!(x < 1.0e9)) return fail(DD_ERR_INVALID_ARG, "shift exceeds 1e9 samples");
        int32_t s = static_cast<int32_t>(std::floor(x + 0.5));  // round half up
        row[c] = s;
        smax = std::max(smax, s);
      }
    }
    rp.s_max = smax;
    rp.gen_n_blocks = static_cast<int32_t>((rp.n_dm + kGenDmPerCta - 1) / kGenDmPerCta);
    rp.gen_span = block_span(rp, n_chan, kGenDmPerCta);

    // Adjoint: channel blocks of kAdjChanBlock (one CTA each), span over the
    // block for each DM: s(last channel) - s(first channel) with shifts
    // non-decreasing towards lower frequency; take the true max/min to allow
    // any order.
    int32_t aspan = 0;
    for (int64_t d = 0; d < rp.n_dm; ++d) {
      const int32_t* row = &rp.shifts[static_cast<size_t>(d) * n_chan];
      for (int32_t c0 = 0; c0 < n_chan; c0 += kAdjChanBlock) {
        int32_t lo = row[c0], hi = row[c0];
        for (int32_t c = c0; c < std::min(c0 + kAdjChanBlock, n_chan); ++c) {
          lo = std::min(lo, row[c]);
          hi = std::max(hi, row[c]);
        }
        aspan = std::max(aspan, hi - lo);
      }
    }
    rp.adj_span = aspan;

    choose_tile(rp, n_chan, p->dtype);
  }
  p->adj.clear();
  if (p->dtype == DD_F32) {
    p->adj.resize(p->ranges.size());
    for (size_t i = 0; i < p->ranges.size(); ++i)
      build_adjoint_range(p->ranges[i], n_chan, &p->adj[i]);
  }
  layout_workspace(p);
  return DD_OK;
}

bool retile_range(dd_plan_s* p, size_t range, int32_t request, int32_t shape_request) {
  RangePlan& rp = p->ranges[range];
  const int32_t old = rp.tile_request, old_shape = rp.shape_request;
  rp.tile_request = request;
  rp.shape_request = shape_request;
  choose_tile(rp, p->n_chan, p->dtype);
  if ((request > 0 || shape_request >= 0) && !rp.tile_ok) {
    rp.tile_request = old;
    rp.shape_request = old_shape;
    choose_tile(rp, p->n_chan, p->dtype);
    layout_workspace(p);
    return false;
  }
  layout_workspace(p);
  return true;
}

}  // namespace dd
