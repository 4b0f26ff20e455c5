/*
 * dd.h -- C ABI of the GB300 brute-force incoherent dedispersion library.
 *
 * The operation (Sec. 2 of the paper, Eq. 3 and Algorithm 1): for every
 * trial DM d of every DM range r and every output sample t,
 *
 *     Y_r[d][t] = sum_{c < n_chan} X_r[c][t + s_r(c, d)]
 *
 * where
 *   - X is a channel-major filterbank X[c][t] (uint8, uint16 or float32),
 *   - X_r is X decimated by the range's time bin b_r (the sum of b_r consecutive
 *     raw samples; the paper's "time binning", Sec. 5.3),
 *   - s_r(c, d) = floor(DM_d * k_c / (b_r * t_samp) + 0.5) is the integer delay
 *     of channel c at trial DM_d = lo_r + d * step_r (fixed step per range,
 *     Table 2), rounded half up, evaluated in FP64 on the host,
 *   - k_c = 4148.808 * (1/f_c^2 - 1/f_ref^2) seconds per unit DM, the
 *     cold-plasma delay law of Eq. 1 in the per-channel form of Eq. 7, with
 *     frequencies in MHz.
 * Outputs are the valid samples only: t in [0, N_out_r) with
 * N_out_r = floor(n_samp / b_r) - S_max_r and S_max_r = max_{c,d} s_r(c, d).
 * Sums are raw (no normalisation): int32 for integer inputs, float32 for float.
 *
 * Memory ownership: the library NEVER allocates device memory.  The caller
 * owns every device buffer (inputs, outputs and the plan workspace); the plan
 * handle itself is host memory owned by the library.  All device work is
 * stream-ordered on the caller's stream, passed as an opaque `void*` holding a
 * cudaStream_t (NULL = the legacy default stream).
 *
 * Errors: every call returns a dd_status; nothing aborts or throws across the
 * boundary.  dd_last_error_detail() gives a thread-local human-readable reason
 * for the last failing call on this thread.  CUDA launch/runtime failures are
 * reported as DD_ERR_CUDA with the CUDA error text in the detail string.
 *
 * Thread safety: a plan is immutable once uploaded; any number of host
 * threads may run it concurrently on different streams.
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DD_OK = 0,
  DD_ERR_INVALID_ARG = 1, /* null pointer, bad enum, non-positive size ... */
  DD_ERR_UNSUPPORTED = 2, /* valid request the library does not implement */
  DD_ERR_SHAPE = 3,       /* input too short, misaligned pointer or stride */
  DD_ERR_BUDGET = 4,      /* workspace or a fixed-size table is too small */
  DD_ERR_CUDA = 5,        /* a CUDA call failed; see dd_last_error_detail() */
  DD_ERR_TIMEOUT = 6      /* a bounded device wait gave up */
} dd_status;

/* Sample types.  DD_U4: 4-bit unsigned samples packed two per byte, the
 * earlier sample in the low nibble; row strides and n_samp still count
 * samples (a row is row_stride / 2 bytes, row_stride a multiple of 32). */
typedef enum { DD_U8 = 1, DD_U16 = 2, DD_F32 = 3, DD_U4 = 4 } dd_dtype;

/* One DM range: trial DMs lo, lo+step, ... (n = llround((hi-lo)/step) of
 * them, half-open like Table 2), dedispersed at time bin `bin` (>= 1). */
typedef struct {
  double dm_lo;
  double dm_hi;
  double dm_step;
  int32_t bin;
} dd_range;

typedef struct dd_plan_s* dd_plan;

#define DD_MAX_RANGES 16

/* Sizes of a plan for a given number of raw input samples. */
typedef struct {
  int32_t n_chan;
  int32_t n_ranges;
  dd_dtype dtype;
  int64_t n_samp;                     /* raw samples the query was made for */
  int64_t n_dm_total;                 /* sum of n_dm over ranges */
  int64_t n_dm[DD_MAX_RANGES];        /* trial DMs per range */
  int64_t s_max[DD_MAX_RANGES];       /* largest shift per range (decimated samples) */
  int64_t n_out[DD_MAX_RANGES];       /* output samples per range (<= 0: too short) */
  int64_t out_offset[DD_MAX_RANGES];  /* element offset of each range in d_out */
  int64_t out_elems;                  /* total output elements */
  int64_t max_delay_raw;              /* max over ranges of (s_max+1)*bin - 1 raw samples */
  size_t workspace_bytes;             /* device workspace dd_plan_upload needs */
  int32_t kernel[DD_MAX_RANGES];      /* forward kernel per range: DD_KERNEL_* */
  int32_t tile_dms[DD_MAX_RANGES];    /* tile of the tiled kernel: DMs per lane,
                                          DD_TILE_PATTERN or DD_TILE_PACKED
                                          (0: generic kernel) */
  int32_t adjoint_kernel;             /* float32 plans: DD_ADJOINT_* dd_run_adjoint
                                          uses (0 for other dtypes) */
  int32_t tile_shape[DD_MAX_RANGES];  /* pattern-tile ranges: the dd_tile_shapes index
                                          in use; -1 for other ranges */
  int32_t packed_copy[DD_MAX_RANGES]; /* 1: the range can run from a packed copy of
                                          the input (DD_TILE_PACKED, or the automatic
                                          pattern tile of uint8, 4-bit or uint16 input
                                          at bin 1, whose tables the packed kernel
                                          also runs) given the scratch of
                                          dd_plan_packed_scratch_bytes; 0 otherwise */
} dd_plan_info;

/* Adjoint kernels (dd_plan_info.adjoint_kernel). */
#define DD_ADJOINT_GATHER 1  /* staged cotangent windows, gathered per channel */
#define DD_ADJOINT_PATTERN 2 /* the forward pattern tile on the cotangent rows with
                                the transposed shift table (channels as trials,
                                shifts s_max - s(c, d)), then expanded over bins */

/* Forward kernels a range can run on (dd_plan_info.kernel). */
#define DD_KERNEL_GENERIC 1 /* shared-memory staged, any dtype and bin */
#define DD_KERNEL_TILED 2   /* TMA-staged register tiles (uint8 at bin 1 in packed 16-bit
                               lanes); bins with bin * sample bytes dividing 16 */

/* Tile code of the pattern family (dd_plan_set_tile, dd_plan_info.tile_dms):
 * 4 DMs per lane, one indexed branch per channel (or channel pair) over the
 * 32 patterns of per-DM shift increments a or a + 1 between a lane's DMs,
 * a = 0..3.  Plans whose shift of some channel grows by more than 4 between
 * consecutive trial DMs cannot use it. */
#define DD_TILE_PATTERN 0x104
/* The pattern tile on a packed copy of uint8, 4-bit, uint16 or float32 input
 * (bin 1): word t of each channel holds samples t and t + 32 H in its 16-bit
 * halves (uint16: sample t widened to 32 bits; float32: a 64-bit word of the
 * two floats, added two at a time), so the staged words are the window words
 * (no unpacking, one barrier per stage).  dd_run
 * writes the copy into caller scratch first: such plans run through
 * dd_run_scratch (dd_plan_input_scratch_bytes sizes it).  The automatic
 * pattern tile of uint8, 4-bit and uint16 input at bin 1 runs the same
 * packed kernel whenever dd_run_scratch is given the scratch of
 * dd_plan_packed_scratch_bytes (full copies or a ring), and the unpacking
 * kernel otherwise. */
#define DD_TILE_PACKED 0x106

/*
 * Build a plan on the host (no device work).  freqs_mhz[n_chan] are channel
 * centre frequencies, each in (0, f_ref_mhz]; conventionally channel 0 is the
 * highest.  t_samp_s > 0 is the raw sampling time.  ranges[n_ranges]
 * (1..DD_MAX_RANGES) each need step > 0, hi > lo >= 0 and bin >= 1.  The
 * library copies what it needs; the caller keeps ownership of freqs and
 * ranges.  On success *out holds a new plan to release with dd_plan_destroy.
 * Errors: DD_ERR_INVALID_ARG for any violated condition above.
 */
dd_status dd_plan_create(const double* freqs_mhz, int32_t n_chan, double f_ref_mhz,
                         double t_samp_s, const dd_range* ranges, int32_t n_ranges,
                         dd_dtype dtype, dd_plan* out);

/* Release a plan (NULL is a no-op).  Device workspace stays the caller's. */
dd_status dd_plan_destroy(dd_plan plan);

/* Fill *out with the plan's sizes for n_samp raw samples (n_samp >= 0). */
dd_status dd_plan_query(dd_plan plan, int64_t n_samp, dd_plan_info* out);

/* Copy the int32 shift table of range `range` to host memory host_out laid
 * out [n_dm][n_chan] (s(c,d) at host_out[d*n_chan + c]). */
dd_status dd_plan_shifts(dd_plan plan, int32_t range, int32_t* host_out);

/*
 * DM plan from a smearing tolerance: the discrete counterpart (fixed step and
 * time bin per range) of an adaptive DM list, as the paper builds for its
 * comparison with adaptive plans (Sec. 5.2).  With the band's lowest and
 * highest channel centres f_lo, f_hi (MHz), channel width df and centre f_c,
 *   t_chan(DM) = 8297.4e3 * DM * df / f_c^3 ms        (Eq. 4, intra-channel smear)
 *   W_b(DM)    = sqrt((b t_samp)^2 + t_chan(DM)^2 + width^2)
 *   k_band     = 4148.808 * (1/f_lo^2 - 1/f_hi^2) s per unit DM   (Eq. 1)
 *   step_b(DM) = 2 W_b(DM) sqrt(tol^2 - 1) / k_band
 * so that a pulse at any DM, at most step/2 from a trial, is broadened by at
 * most a factor tol.  Range r starts at the previous range's end with bin b_r
 * and step step_b(lo_r) (W grows with DM, so the step holds over the range)
 * and ends where the continuous step has doubled, where t_chan reaches 2 b_r
 * t_samp (the next range then bins by 2 b_r, up to max_bin), or at dm_max;
 * its end is rounded up to a whole number of steps (the last range's to half a
 * step past dm_max, so every DM up to dm_max has a trial within step / 2).  The last of max_ranges
 * ranges runs to dm_max.  Writes *n_ranges <= max_ranges (<= DD_MAX_RANGES)
 * ranges.  Errors: DD_ERR_INVALID_ARG (n_chan < 2, tol <= 1, dm_max <= 0,
 * t_samp <= 0, width < 0, max_bin < 1, max_ranges < 1).
 */
dd_status dd_plan_dm_ranges(const double* freqs_mhz, int32_t n_chan, double t_samp_s,
                            double dm_max, double tol, double width_s, int32_t max_bin,
                            int32_t max_ranges, dd_range* out, int32_t* n_ranges);

/*
 * Choose the tile of range `range`: `tile` is the offset tile's DM count per
 * lane (8, 6, 4, 2 or 1), DD_TILE_PATTERN, DD_TILE_PACKED, or 0 = automatic.  Per-plan tile
 * choice follows the paper's per-telescope tuning of D_dm / N_REG (Sec. 4.1).
 * Rebuilds the plan's device tables, so it must be followed by
 * dd_plan_upload (workspace_bytes may change); the plan is unbound until then.
 * Errors: DD_ERR_INVALID_ARG for another code; DD_ERR_UNSUPPORTED if that
 * tile cannot serve the range (unsupported bin, DM offsets or increments too
 * wide for it, window too large for shared memory); the previous choice (and its workspace binding) is
 * kept.
 */
dd_status dd_plan_set_tile(dd_plan plan, int32_t range, int32_t tile);

/*
 * Copy the plan's device tables into caller-owned device memory d_workspace
 * of `bytes` >= workspace_bytes (16-byte aligned), asynchronously on
 * `stream`, and bind that workspace to the plan.  The workspace must stay
 * alive and unmodified while runs are in flight.  The host staging copy lives
 * in the plan, so the plan must outlive the copy (synchronise the stream
 * before destroying a plan whose upload may still be running).  Plans with
 * uint8 or 4-bit pattern tiles also keep their kernels' widening slots in
 * the workspace (320 slots after the tables, 121 MB for 64-DM blocks at
 * H = 23: each CTA widens its 16-bit partial sums into a slot it takes for
 * the duration of a work unit, so runs of one plan on several streams may
 * overlap); only the tables and the slots' flags are copied.
 * Errors: DD_ERR_BUDGET if bytes is too small, DD_ERR_SHAPE if misaligned,
 * DD_ERR_CUDA if the copy cannot be enqueued.
 */
dd_status dd_plan_upload(dd_plan plan, void* d_workspace, size_t bytes, void* stream);

/*
 * Forward transform (Eq. 3) of every range.
 *   d_in:  device, channel-major [n_chan][in_row_stride] elements of the plan
 *          dtype; n_samp <= in_row_stride valid samples per row; 16-byte
 *          aligned base and in_row_stride*elem_size a multiple of 16 bytes.
 *   d_out: device, the concatenation over ranges of [n_dm_r][n_out_r]
 *          (offsets from dd_plan_query), int32 for integer dtypes and float32
 *          for DD_F32; overwritten.  16-byte aligned.
 * Needs a bound workspace (dd_plan_upload).  Asynchronous on `stream`.
 * Errors: DD_ERR_SHAPE if some range has n_out <= 0 or alignment/stride rules
 * are broken, DD_ERR_INVALID_ARG for null pointers or no workspace,
 * DD_ERR_CUDA on a launch failure.
 */
dd_status dd_run(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                 void* d_out, void* stream);

/*
 * Device scratch bytes dd_run_scratch needs for n_samp raw samples: the packed
 * copy of the input, n_chan x ceil4(n_samp) 32-bit words, when some range is
 * on DD_TILE_PACKED; 0 otherwise.  Host only.
 * Errors: DD_ERR_INVALID_ARG for null pointers, DD_ERR_SHAPE for n_samp <= 0.
 */
dd_status dd_plan_input_scratch_bytes(dd_plan plan, int64_t n_samp, size_t* bytes);

/*
 * Device scratch bytes with which dd_run_scratch runs every range that has a
 * packed copy (dd_plan_info.packed_copy) from packed words, for n_samp raw
 * samples.  n_segments = 1: the full copies (one pass packs the whole input,
 * then the ranges' kernels run).  n_segments in [2, 256]: a ring of two
 * slots, each the packed words of one of n_segments time segments of the
 * outputs plus the ranges' largest delay (about 2 (n_out / n_segments +
 * s_max) words per channel): segment k is packed while the kernels of
 * segment k - 1 run, so packing overlaps the transform and the scratch is a
 * fraction of the input's packed size.  0 if no range has a packed copy.
 * Host only.
 * Errors: DD_ERR_INVALID_ARG for null pointers or n_segments outside
 * [1, 256], DD_ERR_SHAPE for n_samp <= 0 or an input shorter than a range's
 * delay, DD_ERR_UNSUPPORTED (n_segments > 1) when the packed ranges need
 * more than one copy or one at a bin above 1 (no ring: give n_segments = 1).
 */
dd_status dd_plan_packed_scratch_bytes(dd_plan plan, int64_t n_samp, int32_t n_segments,
                                       size_t* bytes);

/*
 * dd_run with caller-owned device scratch (16-byte aligned; the library
 * allocates no device memory).  With at least dd_plan_packed_scratch_bytes(1)
 * every range with a packed copy reads the copy written there first (one
 * pass over the input, on `stream`).  With less, but at least the ring of
 * some segment count in [2, 256] (dd_plan_packed_scratch_bytes), those
 * ranges run from the ring with the fewest segments that fits, packing and
 * the segments' kernels overlapped on the plan's own side streams (a
 * high-priority packing stream and a second compute stream, created at the
 * first such call, joined back into `stream`); the other ranges read d_in.
 * With less still, ranges on DD_TILE_PACKED read their full copies (at least
 * dd_plan_input_scratch_bytes) and the others d_in.  The results are the
 * same in every case.  The scratch is in use until the call's work on
 * `stream` completes.  dd_run on a plan with a DD_TILE_PACKED range returns
 * DD_ERR_UNSUPPORTED.
 * Errors: as dd_run; DD_ERR_BUDGET if the scratch is missing or too small
 * for the DD_TILE_PACKED ranges, DD_ERR_SHAPE if it is misaligned.
 */
dd_status dd_run_scratch(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                         void* d_out, void* d_scratch, size_t scratch_bytes, void* stream);

/*
 * The two halves of dd_run_scratch with full copies, for callers that reuse
 * one packed copy (several plans over the same input) or time the transform
 * alone.  dd_pack_input writes the packed copies of d_in into d_scratch:
 * those of every range with a packed copy when scratch_bytes is at least
 * dd_plan_packed_scratch_bytes(1), else those of the DD_TILE_PACKED ranges
 * (sizes and rules as dd_run_scratch; nothing is written when no range reads
 * a copy).  dd_run_packed is dd_run_scratch without the packing pass and
 * never takes the ring: d_scratch (the same scratch_bytes) must hold the
 * copies of the same d_in and n_samp, made by dd_pack_input with a plan of
 * the same channels and tiles.
 * Errors: as dd_run_scratch; dd_pack_input: DD_ERR_UNSUPPORTED if the plan's
 * packed ranges need different copies.
 */
dd_status dd_pack_input(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                        void* d_scratch, size_t scratch_bytes, void* stream);
dd_status dd_run_packed(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                        void* d_out, const void* d_scratch, size_t scratch_bytes, void* stream);

/*
 * dd_run_scratch restricted to a window of outputs: the first n_keep[r]
 * outputs of each range r (1 <= n_keep[r] <= n_out_r), t in [0, n_keep[r]),
 * each equal to that output of dd_run (Eq. 3 evaluated at those t only).
 * d_out receives, for each range in order, n_dm_r rows of n_keep[r] samples
 * (row d at element offset sum_{q<r} n_dm_q n_keep[q] + d n_keep[r]); int32
 * or float32 as dd_run.  The work is proportional to sum_r n_dm_r n_keep[r]:
 * a streaming caller whose window holds the max-delay overlap plus a new
 * chunk asks each range for the chunk's chunk / b_r new outputs only (the
 * real-time processing of Sec. 5.4 done incrementally).  Scratch rules as
 * dd_run_scratch.  n_keep is host memory, read during the call.
 * Errors: as dd_run_scratch; DD_ERR_INVALID_ARG for a NULL n_keep,
 * DD_ERR_SHAPE for an n_keep[r] outside [1, n_out_r].
 */
dd_status dd_run_window(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                        const int64_t* n_keep, void* d_out, void* d_scratch, size_t scratch_bytes,
                        void* stream);

/*
 * Adjoint (transpose) of dd_run for float32 plans: re-dispersion
 *   xbar[c][t] = sum_r sum_d ybar_r[d][floor(t/b_r) - s_r(c, d)]
 * over terms with 0 <= floor(t/b_r) - s_r(c,d) < n_out_r, computed as a gather
 * (no atomics).  d_ybar has dd_run's output layout; d_xbar is device
 * [n_chan][xbar_row_stride] float32, fully overwritten for t < n_samp (samples
 * no output reads get 0).  This operation is this library's own (the paper has
 * no adjoint); it is the derivative of Eq. 3 with respect to X.
 * This call runs the gather kernel (DD_ADJOINT_GATHER) and needs no scratch;
 * dd_run_adjoint_scratch runs the faster pattern kernel where the plan has it.
 * Errors: DD_ERR_UNSUPPORTED for integer plans, otherwise as dd_run.
 */
dd_status dd_run_adjoint(dd_plan plan, const float* d_ybar, float* d_xbar, int64_t n_samp,
                         int64_t xbar_row_stride, void* stream);

/*
 * Device scratch bytes dd_run_adjoint_scratch needs for n_samp raw samples:
 * the padded cotangent rows, max_r 2 n_dm_r x (ceil(n_samp/b_r) + s_max_r)
 * floats (as float pairs; n_dm_r x ... floats where a range's adjoint tile
 * stages single floats), plus the per-range results, sum_r n_chan x
 * ceil(n_samp/b_r) floats, except for a plan of one range at bin 1, whose
 * result goes straight into xbar (rows rounded up to 4 elements); 0 when the
 * plan's adjoint kernel (dd_plan_info.adjoint_kernel) is the gather.  Host
 * only.
 * Errors: DD_ERR_INVALID_ARG for null pointers, DD_ERR_UNSUPPORTED for integer
 * plans, DD_ERR_SHAPE for n_samp <= 0.
 */
dd_status dd_adjoint_scratch_bytes(dd_plan plan, int64_t n_samp, size_t* bytes);

/*
 * dd_run_adjoint with caller-owned device scratch (16-byte aligned; the
 * library allocates no device memory): with at least
 * dd_adjoint_scratch_bytes bytes and a plan whose adjoint_kernel is
 * DD_ADJOINT_PATTERN it runs the forward pattern tile on the cotangent rows
 * (padded into the scratch) with the transposed shift table, then expands
 * the result over each range's time bin; otherwise the gather.  The scratch
 * is in use until the call's work on `stream` completes.
 * Errors: as dd_run_adjoint; DD_ERR_SHAPE for a misaligned scratch.
 */
dd_status dd_run_adjoint_scratch(dd_plan plan, const float* d_ybar, float* d_xbar,
                                 int64_t n_samp, int64_t xbar_row_stride, void* d_scratch,
                                 size_t scratch_bytes, void* stream);

/*
 * Device status of a plan's earlier runs: synchronises `stream`, then returns
 * DD_ERR_TIMEOUT (and clears the flag) if a kernel of this plan gave up a
 * bounded wait since the last call, DD_OK otherwise.  Kernels never trap or
 * spin forever; a timeout leaves that run's output undefined.
 */
dd_status dd_plan_device_status(dd_plan plan, void* stream);

/*
 * Shapes of the pattern tiles, the tuning space of DD_TILE_PATTERN and
 * DD_TILE_PACKED ranges.  The paper tunes its kernel's tile parameters per
 * telescope and plan (Sec. 4.1: the register tile D_dm x D_t and the channels
 * staged per step); these are the same parameters of this library's tiles.
 */
typedef struct {
  int32_t words_per_lane;     /* H: window words a lane holds per trial DM (a
                                 word holds two samples for uint8, 4-bit and
                                 float pairs) */
  int32_t dms_per_lane;       /* trial DMs per lane (4) */
  int32_t warps;              /* warps per CTA */
  int32_t channels_per_stage; /* channels staged per pipeline step */
  int32_t channel_pairs;      /* 1: two channels per add (integer samples) */
  int32_t float_pairs;        /* 1: 64-bit words of two floats (float32 packed tile) */
  int32_t automatic;          /* 1: the automatic choice may take it (else only
                                 dd_plan_set_tile_shape does) */
} dd_tile_shape;

/* Copy up to max_shapes entries of the shape table to out and set *n_shapes
 * to its length (host only; out may be NULL when max_shapes is 0).
 * Errors: DD_ERR_INVALID_ARG for NULL pointers. */
dd_status dd_tile_shapes(dd_tile_shape* out, int32_t max_shapes, int32_t* n_shapes);

/*
 * dd_plan_set_tile for DD_TILE_PATTERN or DD_TILE_PACKED with one explicit
 * shape (an index of dd_tile_shapes; -1: the automatic shape), the
 * autotuner's knob.  Rebuilds the tables (dd_plan_upload
 * follows, as for dd_plan_set_tile).
 * Errors: DD_ERR_INVALID_ARG for another tile or index; DD_ERR_UNSUPPORTED if
 * the shape cannot serve the range (its kind, window or increments), the
 * previous choice and its binding kept.
 */
dd_status dd_plan_set_tile_shape(dd_plan plan, int32_t range, int32_t tile, int32_t shape);

/*
 * Bound of the plan's device waits.  Every kernel stage waits for its copies
 * with at most max_polls polls of the mbarrier (max_polls <= 0: the default,
 * 2^22); a wait that runs out makes the kernel record DD_ERR_TIMEOUT for
 * dd_plan_device_status (or dd_batch_status, or dd_run_u8_noalloc_status),
 * let its issued copies land and return, leaving that run's output undefined;
 * the context stays usable.  hold_stage >= 0 is a test hook for that path: the
 * copies of channel stage hold_stage (of every CTA of the register-tiled
 * kernels) are never issued, so the first wait on it runs out; -1 turns it
 * off.  Host only; takes effect at the next launch (batches: at the next
 * dd_batch_bind).  The paper has no counterpart: the kernels' waits are this
 * library's own.
 * Errors: DD_ERR_INVALID_ARG for a NULL plan or hold_stage < -1.
 */
dd_status dd_plan_set_wait_limit(dd_plan plan, int32_t max_polls, int32_t hold_stage);

/*
 * Front end: time-major samples d_in[t][c] (the order a receiver or a SIGPROC
 * filterbank delivers; row stride in_row_stride >= n_chan elements) to the
 * channel-major rows d_out[c][t] the transform reads (row stride
 * out_row_stride elements), for t in [t_begin, t_end) and c < n_chan; other
 * elements of d_out are not written.  Both buffers 16-byte aligned with
 * 16-byte multiple row strides, t_begin a multiple of 4 / sample bytes,
 * t_end <= out_row_stride.  Exact (a permutation); asynchronous on `stream`.
 * The paper's pipeline transposes its input before dedispersion (Sec. 5.4).
 * Errors: DD_ERR_INVALID_ARG, DD_ERR_SHAPE.
 */
dd_status dd_transpose(dd_dtype dtype, const void* d_in, int64_t in_row_stride, int32_t n_chan,
                       void* d_out, int64_t out_row_stride, int64_t t_begin, int64_t t_end,
                       void* stream);

/*
 * dd_run_host for time-major host input h_in[t][c] (row stride in_row_stride
 * >= n_chan): each segment is copied to the time-major staging buffer
 * d_tm_stage (same layout as h_in), transposed into the channel-major staging
 * buffer d_cm_stage (row stride cm_row_stride >= n_samp) and dedispersed, with
 * the same overlap of copies and kernels as dd_run_host.
 */
dd_status dd_run_host_tmajor(dd_plan plan, const void* h_in, int64_t in_row_stride,
                             int64_t n_samp, void* h_out, void* d_tm_stage, void* d_cm_stage,
                             int64_t cm_row_stride, void* d_out_stage, void* stream);

/*
 * End-to-end forward from HOST buffers: copies h_in (pinned host memory,
 * [n_chan][in_row_stride]) to the caller's device staging buffer d_in_stage,
 * computes the transform into d_out_stage and copies the output planes back to
 * h_out (pinned, the dd_run output layout).  The raw time axis is split into
 * 16 segments: segment k's copy in, the outputs whose dispersion tracks end in
 * segments 0..k, and their copy out run on internal copy streams and on
 * `stream` alternating with an internal compute stream, so copies overlap the
 * kernels.  The internal streams and events
 * are created on the first call (per device) and released by dd_plan_destroy;
 * concurrent calls enqueue one after the other.  When `stream` completes,
 * h_out is written.  Staging buffers have the same
 * layout rules as dd_run.  Returns once the work is enqueued.
 */
dd_status dd_run_host(dd_plan plan, const void* h_in, int64_t in_row_stride, int64_t n_samp,
                      void* h_out, void* d_in_stage, void* d_out_stage, void* stream);

/*
 * dd_run_host with caller-owned device scratch for ranges on DD_TILE_PACKED
 * (16-byte aligned, at least dd_plan_input_scratch_bytes): each segment's
 * columns are packed on an internal stream once the samples 32 H further on
 * have arrived, and those ranges take the outputs whose packed words are
 * complete.  dd_run_host (and dd_run_host_tmajor) return DD_ERR_UNSUPPORTED
 * for such plans.
 * Errors: as dd_run_host; DD_ERR_BUDGET for missing or too little scratch,
 * DD_ERR_SHAPE for a misaligned one.
 */
dd_status dd_run_host_scratch(dd_plan plan, const void* h_in, int64_t in_row_stride,
                              int64_t n_samp, void* h_out, void* d_in_stage, void* d_out_stage,
                              void* d_scratch, size_t scratch_bytes, void* stream);

/*
 * Forward transform of a uint8 plan without any caller-provided workspace, for
 * callers that cannot allocate device memory (for example a real-time
 * pipeline that must not call cudaMalloc while data streams in, or a plug-in
 * whose host framework owns every device allocation).  The paper has no
 * counterpart: it exists only for those callers.
 *   - The plan's tables live in a fixed array of 8 MiB in this library's own
 *     device memory (every GPU that loads the library reserves it until the
 *     process exits).  Plans whose tables exceed it get DD_ERR_BUDGET.
 *   - Every range must run on the tiled kernel (dd_plan_query's kernel is
 *     DD_KERNEL_TILED) and not on DD_TILE_PACKED, otherwise
 *     DD_ERR_UNSUPPORTED.
 *   - d_in / in_row_stride / n_samp / d_out follow dd_run; the plan needs no
 *     dd_plan_upload.  The call allocates nothing and frees nothing.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current).  The address is cached for the life
 *     of the process: cudaDeviceReset between calls is not supported.
 *   - All calls share the one array, which keeps the last call's contents;
 *     each call copies its tables in on `stream` first.  Calls that overlap on
 *     the GPU (different streams, or host threads) race on the array and give
 *     undefined results: serialise them.
 *   - The array starts with a status word, zero when the library loads; a
 *     bounded device wait that gives up sets it (and leaves that call's output
 *     undefined) and dd_run_u8_noalloc_status reads and clears it.
 */
dd_status dd_run_u8_noalloc(dd_plan plan, const void* d_in, int64_t in_row_stride,
                            int64_t n_samp, void* d_out, void* stream);

/*
 * Wait status of the dd_run_u8_noalloc calls on the current device since the
 * last check: synchronises `stream`, returns DD_ERR_TIMEOUT (and clears the
 * status word) if a bounded device wait of one of them gave up, DD_OK
 * otherwise.  Reads the word in the fixed array through the address cached by
 * the first dd_run_u8_noalloc call (DD_OK if there was none); allocates
 * nothing.  The paper has no counterpart.
 * Errors: DD_ERR_CUDA if the copy or the synchronisation fails.
 */
dd_status dd_run_u8_noalloc_status(void* stream);

/* ---------------------------------------------------------------------------
 * Persistent batches: many beams (plans of different channel counts, dtypes,
 * sampling times and DM plans) dedispersed by persistent launches of the
 * tiled kernels -- one for the ranges on the pattern tile, one for those on
 * offset tiles -- whose CTAs take (beam range, DM block, time tile) work items
 * from a device counter, longest items first.  The paper tunes its tile
 * parameters per telescope and plan (Sec. 4.1); here each plan's tile is
 * chosen before the batch is built (dd_plan_set_tile), so the batch mixes
 * tiles.  The batch keeps pointers to its plans, which must outlive it and
 * stay uploaded.  Device memory is the caller's (dd_batch_workspace_bytes).
 * ------------------------------------------------------------------------- */
typedef struct dd_batch_s* dd_batch;

/* Build the work lists for n_plans plans and their raw sample counts.  Every
 * range must be on the tiled kernel, on the pattern tile (DD_TILE_PACKED
 * included) or an offset tile with 4, 2 or 1 DMs per lane, else
 * DD_ERR_UNSUPPORTED; DD_ERR_BUDGET if the plans' windows together exceed the
 * persistent kernel's shared memory; DD_ERR_SHAPE if an input is shorter than
 * a range's maximum delay. */
dd_status dd_batch_create(const dd_plan* plans, const int64_t* n_samp, int32_t n_plans,
                          dd_batch* out);
dd_status dd_batch_destroy(dd_batch batch);
/* Device workspace bytes the batch needs (work counter, job table, items). */
dd_status dd_batch_workspace_bytes(dd_batch batch, size_t* bytes);
/* Number of work items and jobs (plan ranges) of the batch. */
dd_status dd_batch_info(dd_batch batch, int64_t* n_items, int32_t* n_jobs);
/* Kernel launches one dd_batch_run makes (one per pattern-tile variant present,
 * one if any range is on an offset tile, and one packing launch per plan with
 * a DD_TILE_PACKED range). */
dd_status dd_batch_launches(dd_batch batch, int32_t* n_launches);
/* Copy the work list into caller device memory (256-byte aligned, >= the
 * workspace bytes) and bind it; synchronises `stream`. */
dd_status dd_batch_upload(dd_batch batch, void* d_workspace, size_t bytes, void* stream);
/* Bind the input/output buffers of every plan (d_in[i], in_row_stride[i],
 * d_out[i] follow dd_run's rules for plan i) by uploading the job table;
 * synchronises `stream`.  Rebind whenever a buffer address changes.
 * Errors: DD_ERR_UNSUPPORTED if a plan has a DD_TILE_PACKED range (bind it with
 * dd_batch_bind_scratch). */
dd_status dd_batch_bind(dd_batch batch, const void* const* d_in, const int64_t* in_row_stride,
                        void* const* d_out, void* stream);
/* Device scratch bytes plan `plan` of the batch needs for its packed copy
 * (dd_plan_input_scratch_bytes at the batch's sample count; 0 without a
 * DD_TILE_PACKED range).  Host only. */
dd_status dd_batch_plan_scratch_bytes(dd_batch batch, int32_t plan, size_t* bytes);
/* dd_batch_bind with caller-owned scratch per plan (d_scratch[i] of
 * scratch_bytes[i] >= dd_batch_plan_scratch_bytes, 16-byte aligned; NULL
 * arrays or entries for plans without a packed range): each dd_batch_run then
 * first writes the packed copies (one packing launch per such plan), and the
 * persistent launches read them.  The scratch is in use while runs are.
 * Errors: as dd_batch_bind; DD_ERR_UNSUPPORTED for missing scratch,
 * DD_ERR_BUDGET for too little, DD_ERR_SHAPE for a misaligned one. */
dd_status dd_batch_bind_scratch(dd_batch batch, const void* const* d_in,
                                const int64_t* in_row_stride, void* const* d_out,
                                void* const* d_scratch, const size_t* scratch_bytes,
                                void* stream);
/* Persistent launches over all items of a bound batch: a counter reset, the
 * packing launches of plans bound with scratch, and one kernel launch per tile
 * family present.  The families run on concurrent lanes (the batch's own
 * streams, created by dd_batch_upload, forked from `stream` after the reset
 * and joined into it at the end), each lane packing the inputs it reads
 * first; all of it can be captured in a CUDA graph from `stream`. */
dd_status dd_batch_run(dd_batch batch, void* stream);
/* DD_ERR_TIMEOUT if a bounded device wait of any batch plan gave up since the
 * last check (clears the flags); synchronises `stream`. */
dd_status dd_batch_status(dd_batch batch, void* stream);

/* Human-readable name of a status code (static storage). */
const char* dd_status_string(dd_status status);
/* Thread-local detail of the last failing call on this thread ("" if none). */
const char* dd_last_error_detail(void);
/* Library version string. */
const char* dd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
