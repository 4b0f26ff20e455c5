// dd_internal.h -- host-side plan representation and kernel launch interfaces
// shared by the translation units of libdd (planner, kernels, C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "dd.h"
#include "fwd_tiled.h"

namespace dd {

// Dispersion constant of the cold-plasma delay law (Eq. 1), MHz^2 s pc^-1 cm^3.
constexpr double kDispersionConstant = 4148.808;

// Tile of the generic forward kernel: DMs per CTA (8 warps x kGenDmPerThread).
constexpr int kGenDmPerThread = 2;
constexpr int kGenSampPerThread = 8;
constexpr int kGenDmPerCta = 8 * kGenDmPerThread;

// Adjoint blocking (adjoint.cu): channels per CTA.
constexpr int kAdjChanBlock = 64;
constexpr int kGenSampPerCta = 32 * kGenSampPerThread;

struct RangePlan {
  dd_range r{};
  int64_t n_dm = 0;
  int32_t s_max = 0;
  std::vector<int32_t> shifts;  // [n_dm][n_chan]

  // Generic kernel blocking.
  int32_t gen_n_blocks = 0;     // DM blocks of kGenDmPerCta
  int32_t gen_span = 0;         // max over blocks/channels of in-block shift span

  // Adjoint blocking: max over channel blocks and DMs of the in-block span.
  int32_t adj_span = 0;

  // Register-tiled kernel (fwd_tiled.cu), used when tile_ok (time bin 1).
  bool tile_ok = false;
  bool tile_pattern = false;    // pattern tile (fwd_pattern.cu) instead of offset tile
  int32_t tile_dr = 0;          // DMs per lane of the chosen tile shape
  int32_t tile_h = 0;           // window words per lane per DM (kH, or the pattern H)
  int32_t tile_shape = 0;       // index into tk::kPatShapes (pattern tiles)
  int32_t tile_kind = 0;        // window-word kind (tk::Kind)
  int32_t tile_request = 0;     // tile requested by dd_plan_set_tile (0 = automatic)
  int32_t shape_request = -1;   // pattern shape requested (dd_plan_set_tile_shape; -1: first fit)
  int32_t tile_n_blocks = 0;    // DM blocks of tile_dr * warps DMs
  int32_t tile_lp = 0;          // window words per staged channel
  uint32_t tile_units_magic = 0;  // division by tile_lp / 4 (see fwd_tiled.h)
  int32_t tile_units_shift = 0;
  size_t tile_chunk_off = 0;    // pair tiles: byte offset of the pair chunks in tile_recs
  int32_t tile_chunk_bytes = 0; // pair tiles: bytes per (DM block, stage) chunk
  int32_t tile_n_chan = 0;      // rows of the tables' input when not the plan's channels
  // Automatic pattern tiles of uint8, 4-bit and uint16 input at time bin 1:
  // the packed-copy kind (kU8P, kU16P) whose kernel runs the same tables
  // from a packed copy of the input (the tables are planned at the plain
  // kind's window alignment, a multiple of the packed kind's); 0 if none.
  int32_t alt_kind = 0;

  // Byte offsets of the device tables inside the workspace.
  size_t off_shifts = 0;        // int32 [n_dm][n_chan]
  size_t off_tile_recs = 0;     // tk::Rec or tk::PRec [tile_n_blocks][n_chan]
  std::vector<unsigned char> tile_recs;  // host image of the records
};


}  // namespace dd

struct dd_plan_s {
  int32_t n_chan = 0;
  double f_ref = 0.0;
  double t_samp = 0.0;
  dd_dtype dtype = DD_U8;
  std::vector<double> freqs;
  std::vector<double> k;  // delay coefficient per channel [s per unit DM]
  std::vector<dd::RangePlan> ranges;
  std::vector<unsigned char> host_ws;  // staged device tables
  void* d_ws = nullptr;                // bound device workspace (caller-owned)
  size_t ws_bytes = 0;
  void* host_pipe = nullptr;           // streams/events of dd_run_host (api.cu)
  // Float32 plans: per range, its adjoint as a forward transform (plan.cpp,
  // build_adjoint_range; tile_ok false where the pattern tile cannot serve it).
  std::vector<dd::RangePlan> adj;
  // Bounded device waits (dd_plan_set_wait_limit): polls before a pipeline
  // wait gives up, and the channel stage whose copies are withheld (-1: none).
  int32_t wait_iters = dd::tk::kWaitIters;
  int32_t hold_stage = -1;
  // Widening slots in the workspace (plan.cpp, layout_workspace): 64-bit
  // words per slot (0: none) and byte offsets of the slot flags and slots.
  // The workspace image (host_ws) ends before the slots: they need no
  // initial contents.
  int32_t wslot_words = 0;
  size_t off_wflags = 0;
  size_t off_wslots = 0;
};

namespace dd {

// Thread-local error detail helpers (api.cu).
dd_status fail(dd_status st, const std::string& detail);
dd_status cuda_fail(int err, const char* what);

// Planner (plan.cpp).
dd_status build_plan(dd_plan_s* p);
// (Re)choose the uint8 tile of one range (request 0 = automatic) and rebuild
// the workspace image.  Returns false if the requested tile does not fit.
bool retile_range(dd_plan_s* p, size_t range, int32_t request, int32_t shape_request = -1);
int64_t range_n_out(const dd_plan_s* p, const RangePlan& rp, int64_t n_samp);
// DM ranges from a smearing tolerance (dd_plan_dm_ranges); returns their count.
int32_t dm_plan_ranges(const double* freqs, int32_t n_chan, double t_samp, double dm_max,
                       double tol, double width, int32_t max_bin, int32_t max_ranges,
                       dd_range* out);

// Kernel launchers (return a cudaError_t as int; 0 on success).  Each writes
// the outputs t in [t_begin, t_end) of rows of n_out samples; t_begin is a
// multiple of range_tile_samples(rp).
int64_t range_tile_samples(const RangePlan& rp);
int launch_forward_generic(const dd_plan_s* p, const RangePlan& rp, const void* d_in,
                           int64_t stride, int64_t n_samp, int64_t n_out, void* d_out,
                           int64_t t_begin, int64_t t_end, void* stream);
int launch_forward_tiled(const dd_plan_s* p, const RangePlan& rp, const void* d_in,
                         int64_t stride, int64_t n_samp, int64_t n_out, void* d_out,
                         int64_t t_begin, int64_t t_end, void* stream);
// The tiled kernel with its record table and status word at explicit device
// addresses (used by the no-allocation entry point and the batch runtime).
// widen_slots = false: the widening never uses the plan workspace's slots
// (the no-allocation entry point, whose plan may have no workspace).
int launch_forward_tiled_with_tables(const dd_plan_s* p, const RangePlan& rp, const void* recs,
                                     int32_t* err, const void* d_in, int64_t stride,
                                     int64_t n_out, void* d_out, int64_t t_begin, int64_t t_end,
                                     void* stream, bool widen_slots = true);
// The pattern kernel (fwd_pattern.cu), same arguments; output row d + 1
// starts out_stride elements after row d (n_out for the output layout of
// dd_run; negative for rows written in reverse order).
// `kind` > 0 runs the tables with that kernel kind (a packed-copy kind the
// range's copy_kind allows) and `x_origin` is the sample held by element 0
// of each input row (a time segment's packed words in a ring slot; a
// multiple of the tables' window alignment).
int launch_forward_pattern(const dd_plan_s* p, const RangePlan& rp, const void* recs,
                           int32_t* err, const void* d_in, int64_t stride, int64_t n_out,
                           void* d_out, int64_t t_begin, int64_t t_end, void* stream,
                           int64_t out_stride, int kind = 0, int64_t x_origin = 0,
                           bool widen_slots = true);
// Packed uint8 copy for the kU8P tiles (pack.cu): out[c][t] = in[c][t] |
// in[c][t + pair] << 16 for t in [t_begin, t_end) (0 past n_samp); strides in
// bytes (in) and 32-bit words (out, a multiple of 4); pair and t_begin
// multiples of 16, t_end of 4.  Source kU4: 4-bit
// input, two samples per byte (the earlier in the low nibble); kU16: uint16
// input widened, out[c][t] = in[c][t] (pair unused); kF32: float32 input,
// 64-bit words out[c][t] = (in[c][t], in[c][t + pair]) (out_stride in those
// words).
enum class PackSource { kU8, kU4, kU16, kF32 };
// out_origin: the word held by element 0 of each output row (a ring slot
// holding words [out_origin, out_origin + out_stride)); t_begin >= out_origin,
// t_end <= out_origin + out_stride, out_origin a multiple of 16.
int launch_pack_pairs(const void* d_in, int64_t in_stride, int32_t n_chan, int64_t n_samp,
                      void* d_out, int64_t out_stride, int32_t pair, int64_t t_begin,
                      int64_t t_end, PackSource src, void* stream, int64_t out_origin = 0);
// uint8 decimated by bin (2, 4, 8) into packed pair words of decimated samples
// (pack.cu): out[c][t] = D[c][t] | D[c][t + pair] << 16, D the sums of bin
// consecutive samples, t < out_stride (a multiple of 4, >= n_samp / bin), 0
// past n_samp / bin; in_stride in bytes.
int launch_pack_pairs_binned(const void* d_in, int64_t in_stride, int32_t n_chan, int64_t n_samp,
                             int32_t bin, void* d_out, int64_t out_stride, int32_t pair,
                             void* stream);
// The kernel kind that runs range rp from a packed copy of the input: its
// own kind on DD_TILE_PACKED, the alternative kind of an automatic pattern
// tile when `with_auto` (the caller's scratch holds copies for those too),
// else 0 (the range reads the input itself).
inline int copy_kind(const RangePlan& rp, bool with_auto) {
  if (!rp.tile_ok || !rp.tile_pattern) return 0;
  if (tk::packed_copy_kind(rp.tile_kind)) return rp.tile_kind;
  return with_auto ? rp.alt_kind : 0;
}
// Pair distance of the packed copy a range reads with kernel kind `kind`.
inline int32_t pack_pair(const RangePlan& rp, int kind) {
  return kind == tk::kU8P || kind == tk::kF32P ? 32 * rp.tile_h : 0;
}
inline int32_t pack_pair(const RangePlan& rp) { return pack_pair(rp, rp.tile_kind); }
inline PackSource pack_source(dd_dtype dtype) {
  return dtype == DD_U16   ? PackSource::kU16
         : dtype == DD_U4  ? PackSource::kU4
         : dtype == DD_F32 ? PackSource::kF32
                           : PackSource::kU8;
}
// The packed copies a plan's DD_TILE_PACKED ranges read (api.cu): one per
// distinct (pair distance, bin), in range order, at 256-byte aligned offsets
// of the caller's scratch; each copy has `stride` words per channel row.
struct PackedCopy {
  int32_t pair;
  int32_t bin;
  int64_t stride;  // words per row: ceil4(n_samp / bin)
  size_t offset;   // bytes into the scratch
  size_t bytes;
};
// The copies, and for each range its copy (-1: reads the input itself);
// with_auto: also the copies of the automatic tiles with an alt_kind.
std::vector<PackedCopy> packed_copies(const dd_plan_s* p, int64_t n_samp,
                                      std::vector<int32_t>* range_copy, bool with_auto = false);
// Bytes all copies take (0 without a packed range).
size_t packed_input_bytes(const dd_plan_s* p, int64_t n_samp, bool with_auto = false);
// Write one copy of the input (in_stride in samples) into scratch.
int launch_pack_copy(const dd_plan_s* p, const PackedCopy& pc, const void* d_in, int64_t in_stride,
                     int64_t n_samp, void* d_scratch, void* stream);
// Bytes of n samples of a dtype (4-bit: two per byte, rounded up).
inline size_t dtype_row_bytes(dd_dtype t, int64_t n) {
  return t == DD_U4    ? static_cast<size_t>((n + 1) / 2)
         : t == DD_U8  ? static_cast<size_t>(n)
         : t == DD_U16 ? static_cast<size_t>(n) * 2
                       : static_cast<size_t>(n) * 4;
}
// Bytes of one word of a plan's packed copy.
inline size_t packed_word_bytes(dd_dtype dtype) { return dtype == DD_F32 ? 8 : 4; }
// Time-major [t][c] to channel-major [c][t] for t in [t_begin, t_end) (transpose.cu).
int launch_transpose(int elem_bytes, const void* d_in, int64_t in_row_stride, int32_t n_chan,
                     void* d_out, int64_t out_row_stride, int64_t t_begin, int64_t t_end,
                     void* stream);
// Adjoint (adjoint.cu): with d_scratch of at least adjoint_scratch_bytes()
// bytes the pattern kernel runs where the plan has its tables, else the gather.
int launch_adjoint(const dd_plan_s* p, const float* d_ybar, float* d_xbar, int64_t n_samp,
                   int64_t stride, const int64_t* n_out, const int64_t* out_off,
                   void* d_scratch, size_t scratch_bytes, void* stream);
// Scratch bytes of the pattern adjoint for n_samp raw samples (0: the plan's
// adjoint is the gather).
size_t adjoint_scratch_bytes(const dd_plan_s* p, int64_t n_samp);

tk::TileParams tiled_params(const dd_plan_s* p, const RangePlan& rp, const void* recs,
                            int32_t* err, const void* d_in, int64_t stride, int64_t n_out,
                            void* d_out, int kind = 0, bool widen_slots = true);
int launch_batch(const tk::BatchArgs& args, int32_t grid, size_t smem, void* stream);
// Per-kind launchers of the pattern kernels (fwd_pattern_k*.cu): the
// one-unit-per-CTA kernel and the persistent batch kernel of kPatShapes[shape].
#define DD_PATTERN_KINDS(X) X(kU8) X(kU8W) X(kU8P) X(kU4) X(kU16) X(kU16P) X(kF32) X(kF32D) X(kF32P)
#define DD_DECLARE_PATTERN_KIND(K)                                                            \
  int pattern_forward_##K(int shape, const tk::TileParams& prm, int64_t grid, void* stream); \
  int pattern_batch_##K(int shape, const tk::PatBatchArgs& args, int32_t grid, size_t smem,  \
                        void* stream, int mode);
DD_PATTERN_KINDS(DD_DECLARE_PATTERN_KIND)
#undef DD_DECLARE_PATTERN_KIND
// Persistent pattern-tile launch of one variant (kind, tk::kPatShapes index);
// mode: the widening mode (tk::widen_mode) every job of the launch takes.
int launch_pattern_batch(int kind, int shape, const tk::PatBatchArgs& args, int32_t grid,
                         size_t smem, void* stream, int mode);

}  // namespace dd
