// api.cu -- the C ABI of libdd (declared in include/dd.h): argument checking,
// error reporting and kernel dispatch.  No device memory is allocated here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "dd_internal.h"

namespace dd {

namespace {
thread_local std::string g_detail;
}

void free_host_pipe(dd_plan_s* p);

dd_status fail(dd_status st, const std::string& detail) {
  g_detail = detail;
  return st;
}

dd_status cuda_fail(int err, const char* what) {
  g_detail = std::string(what) + ": " + cudaGetErrorName(static_cast<cudaError_t>(err)) +
             " (" + cudaGetErrorString(static_cast<cudaError_t>(err)) + ")";
  return DD_ERR_CUDA;
}

std::vector<PackedCopy> packed_copies(const dd_plan_s* p, int64_t n_samp,
                                      std::vector<int32_t>* range_copy, bool with_auto) {
  std::vector<PackedCopy> copies;
  if (range_copy) range_copy->assign(p->ranges.size(), -1);
  size_t off = 0;
  for (size_t r = 0; r < p->ranges.size(); ++r) {
    const RangePlan& rp = p->ranges[r];
    const int kind = copy_kind(rp, with_auto);
    if (kind == 0) continue;
    const int32_t pair = pack_pair(rp, kind), bin = rp.r.bin;
    size_t k = 0;
    while (k < copies.size() && !(copies[k].pair == pair && copies[k].bin == bin)) ++k;
    if (k == copies.size()) {
      PackedCopy pc{};
      pc.pair = pair;
      pc.bin = bin;
      pc.stride = (std::max<int64_t>(n_samp / bin, 1) + 3) / 4 * 4;
      pc.offset = off;
      pc.bytes = static_cast<size_t>(p->n_chan) * static_cast<size_t>(pc.stride) *
                 packed_word_bytes(p->dtype);
      off = (off + pc.bytes + 255) / 256 * 256;
      copies.push_back(pc);
    }
    if (range_copy) (*range_copy)[r] = static_cast<int32_t>(k);
  }
  return copies;
}

size_t packed_input_bytes(const dd_plan_s* p, int64_t n_samp, bool with_auto) {
  const auto copies = packed_copies(p, n_samp, nullptr, with_auto);
  return copies.empty() ? 0 : copies.back().offset + copies.back().bytes;
}

int launch_pack_copy(const dd_plan_s* p, const PackedCopy& pc, const void* d_in, int64_t in_stride,
                     int64_t n_samp, void* d_scratch, void* stream) {
  unsigned char* dst = static_cast<unsigned char*>(d_scratch) + pc.offset;
  const int64_t in_bytes = static_cast<int64_t>(dtype_row_bytes(p->dtype, in_stride));
  if (pc.bin > 1)
    return launch_pack_pairs_binned(d_in, in_bytes, p->n_chan, n_samp, pc.bin, dst, pc.stride,
                                    pc.pair, stream);
  return launch_pack_pairs(d_in, in_bytes, p->n_chan, n_samp, dst, pc.stride, pc.pair, 0,
                           pc.stride, pack_source(p->dtype), stream);
}

namespace {

size_t elem_size(dd_dtype t) { return (t == DD_U8 || t == DD_U4) ? 1 : (t == DD_U16 ? 2 : 4); }
// Bytes of n samples of a dtype (4-bit: two per byte, rounded up).
size_t row_bytes(dd_dtype t, int64_t n) {
  return t == DD_U4 ? static_cast<size_t>((n + 1) / 2) : static_cast<size_t>(n) * elem_size(t);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

dd_status fill_info(const dd_plan_s* p, int64_t n_samp, dd_plan_info* o) {
  std::memset(o, 0, sizeof(*o));
  o->n_chan = p->n_chan;
  o->n_ranges = static_cast<int32_t>(p->ranges.size());
  o->dtype = p->dtype;
  o->n_samp = n_samp;
  int64_t off = 0;
  for (size_t i = 0; i < p->ranges.size(); ++i) {
    const RangePlan& rp = p->ranges[i];
    o->n_dm[i] = rp.n_dm;
    o->s_max[i] = rp.s_max;
    o->n_out[i] = range_n_out(p, rp, n_samp);
    o->out_offset[i] = off;
    if (o->n_out[i] > 0) off += rp.n_dm * o->n_out[i];
    o->n_dm_total += rp.n_dm;
    o->kernel[i] = rp.tile_ok ? DD_KERNEL_TILED : DD_KERNEL_GENERIC;
    o->tile_shape[i] = rp.tile_ok && rp.tile_pattern ? rp.tile_shape : -1;
    o->packed_copy[i] = copy_kind(rp, true) != 0 ? 1 : 0;
    o->tile_dms[i] = !rp.tile_ok                          ? 0
                     : !rp.tile_pattern                   ? rp.tile_dr
                     : tk::packed_copy_kind(rp.tile_kind)  ? DD_TILE_PACKED
                                                           : DD_TILE_PATTERN;
    int64_t raw = (static_cast<int64_t>(rp.s_max) + 1) * rp.r.bin - 1;
    if (raw > o->max_delay_raw) o->max_delay_raw = raw;
  }
  o->out_elems = off;
  o->workspace_bytes = p->ws_bytes;
  o->adjoint_kernel = 0;
  if (p->dtype == DD_F32) {
    bool all = !p->adj.empty();
    for (const auto& ar : p->adj) all = all && ar.tile_ok;
    o->adjoint_kernel = all && p->n_chan <= 65535 ? DD_ADJOINT_PATTERN : DD_ADJOINT_GATHER;
  }
  return DD_OK;
}

// dd_run_host splits the raw time axis into this many segments: segment k's
// host-to-device copy, the outputs it completes and their device-to-host copy
// run on separate streams, overlapping segment k+1's copy in and k-1's copy
// out.  Segments alternate between two compute streams (the caller's and an
// internal one) so that one segment's last CTAs overlap the next one's first.
constexpr int kHostSegments = 16;

// Slots of the packed ring (dd_run_scratch with less scratch than the full
// packed copies): segment k is packed into slot k % kRingSlots while the
// kernels of segment k - 1 run.
constexpr int kRingSlots = 2;
constexpr int kRingMaxSegments = 256;

struct HostPipe {
  int device = -1;
  cudaStream_t s_in = nullptr, s_out = nullptr, s_comp = nullptr, s_tr = nullptr;
  cudaStream_t s_pack = nullptr;  // ring packing, at the highest stream priority
  cudaEvent_t start = nullptr, done = nullptr;
  cudaEvent_t in[kHostSegments] = {}, comp[kHostSegments] = {}, tr[kHostSegments] = {};
  cudaEvent_t packed[kRingSlots] = {}, freed[kRingSlots] = {};
};

// The plans' side streams and events are shared by every call on a plan:
// calls from several host threads enqueue one after the other (each wait
// captures the record of its own call).
std::mutex g_pipe_mu;

void destroy_pipe(HostPipe* hp) {
  if (hp->s_in) cudaStreamDestroy(hp->s_in);
  if (hp->s_out) cudaStreamDestroy(hp->s_out);
  if (hp->s_comp) cudaStreamDestroy(hp->s_comp);
  if (hp->s_tr) cudaStreamDestroy(hp->s_tr);
  if (hp->s_pack) cudaStreamDestroy(hp->s_pack);
  for (cudaEvent_t e : {hp->start, hp->done})
    if (e) cudaEventDestroy(e);
  for (int k = 0; k < kRingSlots; ++k) {
    if (hp->packed[k]) cudaEventDestroy(hp->packed[k]);
    if (hp->freed[k]) cudaEventDestroy(hp->freed[k]);
  }
  for (int k = 0; k < kHostSegments; ++k) {
    if (hp->in[k]) cudaEventDestroy(hp->in[k]);
    if (hp->comp[k]) cudaEventDestroy(hp->comp[k]);
    if (hp->tr[k]) cudaEventDestroy(hp->tr[k]);
  }
  delete hp;
}

// The plan's copy streams and events on the current device (created once).
cudaError_t host_pipe(dd_plan_s* p, HostPipe** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  HostPipe* hp = static_cast<HostPipe*>(p->host_pipe);
  if (hp && hp->device == dev) {
    *out = hp;
    return cudaSuccess;
  }
  if (hp) destroy_pipe(hp);
  p->host_pipe = nullptr;
  hp = new (std::nothrow) HostPipe();
  if (!hp) return cudaErrorMemoryAllocation;
  hp->device = dev;
  e = cudaStreamCreateWithFlags(&hp->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->s_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->s_tr, cudaStreamNonBlocking);
  int prio_least = 0, prio_greatest = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&hp->s_pack, cudaStreamNonBlocking, prio_greatest);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->done, cudaEventDisableTiming);
  for (int k = 0; k < kRingSlots && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&hp->packed[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->freed[k], cudaEventDisableTiming);
  }
  for (int k = 0; k < kHostSegments && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&hp->in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->comp[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->tr[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    destroy_pipe(hp);
    return e;
  }
  p->host_pipe = hp;
  *out = hp;
  return cudaSuccess;
}

// A failure after the side streams were forked from the caller's stream:
// the caller's stream still waits for whatever they already hold (as far as
// the calls still succeed), so that the caller's next use of its buffers
// cannot overtake copies or kernels queued there.
dd_status fail_joined(HostPipe* hp, cudaStream_t s, int err, const char* what) {
  for (cudaStream_t o : {hp->s_in, hp->s_out, hp->s_comp, hp->s_tr, hp->s_pack})
    if (cudaEventRecord(hp->done, o) == cudaSuccess) cudaStreamWaitEvent(s, hp->done, 0);
  return cuda_fail(err, what);
}

}  // namespace

void free_host_pipe(dd_plan_s* p) {
  if (p->host_pipe) destroy_pipe(static_cast<HostPipe*>(p->host_pipe));
  p->host_pipe = nullptr;
}

namespace {


// Outputs [t_begin, t_end) of range rp.  kind > 0: the pattern tables run
// by that packed-copy kernel (copy_kind) on packed words, element 0 of each
// row holding word x_origin.
int launch_range(const dd_plan_s* p, const RangePlan& rp, const void* d_in, int64_t stride,
                 int64_t n_samp, int64_t n_out, void* d_out, int64_t t_begin, int64_t t_end,
                 void* stream, int kind = 0, int64_t x_origin = 0) {
  if (kind > 0) {
    unsigned char* ws = static_cast<unsigned char*>(p->d_ws);
    return launch_forward_pattern(p, rp, ws + rp.off_tile_recs,
                                  reinterpret_cast<int32_t*>(ws + tk::kStatusOffset), d_in,
                                  stride, n_out, d_out, t_begin, t_end, stream, n_out, kind,
                                  x_origin);
  }
  return rp.tile_ok ? launch_forward_tiled(p, rp, d_in, stride, n_samp, n_out, d_out, t_begin,
                                           t_end, stream)
                    : launch_forward_generic(p, rp, d_in, stride, n_samp, n_out, d_out, t_begin,
                                             t_end, stream);
}

// The full packed copies a run reads: those of every range with a copy
// kind, automatic tiles included, when the scratch holds them all (and
// they add to the DD_TILE_PACKED ranges' copies); else the DD_TILE_PACKED
// ranges' only.
bool full_with_auto(const dd_plan_s* p, int64_t n_samp, const void* d_scratch, size_t bytes) {
  if (!d_scratch) return false;
  const size_t all = packed_input_bytes(p, n_samp, true);
  return all > packed_input_bytes(p, n_samp, false) && bytes >= all;
}

// One time segment of the ring: packed words [origin, end) in its slot, and
// the outputs [lo_r, hi_r) each ring range computes from them.
struct RingSeg {
  int64_t origin = 0;
  int64_t end = 0;
  int64_t lo[DD_MAX_RANGES] = {};
  int64_t hi[DD_MAX_RANGES] = {};
};
struct RingLayout {
  int32_t pair = 0;
  int64_t slot_words = 0;     // words per channel row of a slot
  size_t slot_bytes = 0;      // a slot, 256-byte aligned
  bool ring[DD_MAX_RANGES] = {};  // the range runs from the ring
  std::vector<RingSeg> segs;  // the segments with work
  size_t bytes() const { return kRingSlots * slot_bytes; }
};

// The ring for n_seg segments of the longest ring range's outputs, each
// range's boundaries rounded down to its time tiles.  False when the ranges
// with a copy kind need more than one copy, or one at a bin above 1 (those
// need the full copies), or there are none.
bool ring_layout(const dd_plan_s* p, const dd_plan_info& info, int64_t n_samp, int n_seg,
                 RingLayout* L) {
  std::vector<int32_t> rc;
  const std::vector<PackedCopy> copies = packed_copies(p, n_samp, &rc, true);
  if (copies.size() != 1 || copies[0].bin != 1 || n_seg < 2) return false;
  *L = RingLayout{};
  L->pair = copies[0].pair;
  int64_t n_max = 0;
  for (size_t r = 0; r < p->ranges.size(); ++r)
    if (rc[r] >= 0) {
      L->ring[r] = true;
      n_max = std::max(n_max, info.n_out[r]);
    }
  const int64_t seg = (n_max + n_seg - 1) / n_seg;
  int64_t words = 0;
  for (int k = 0; k < n_seg; ++k) {
    RingSeg sg;
    int64_t lo_min = -1, need = 0;
    for (size_t r = 0; r < p->ranges.size(); ++r) {
      if (!L->ring[r]) continue;
      const RangePlan& rp = p->ranges[r];
      const int64_t ts = range_tile_samples(rp), n_out = info.n_out[r];
      const int64_t lo = std::min(n_out, k * seg / ts * ts);
      const int64_t hi = k == n_seg - 1 ? n_out : std::min(n_out, (k + 1) * seg / ts * ts);
      sg.lo[r] = lo;
      sg.hi[r] = hi;
      if (hi <= lo) continue;
      lo_min = lo_min < 0 ? lo : std::min(lo_min, lo);
      // Output t reads packed words t' <= t + s_max (a packed word t' holds
      // samples t' and t' + pair).
      need = std::max(need, hi + static_cast<int64_t>(rp.s_max));
    }
    if (lo_min < 0) continue;
    sg.origin = lo_min / 32 * 32;  // a multiple of every tables' window alignment
    sg.end = std::min(copies[0].stride, (need + 15) / 16 * 16);
    words = std::max(words, sg.end - sg.origin);
    L->segs.push_back(sg);
  }
  L->slot_words = (words + 15) / 16 * 16;
  L->slot_bytes = (static_cast<size_t>(p->n_chan) * static_cast<size_t>(L->slot_words) *
                       packed_word_bytes(p->dtype) + 255) / 256 * 256;
  return !L->segs.empty();
}

// The fewest segments (at least 2) whose ring fits `bytes`.
bool pick_ring(const dd_plan_s* p, const dd_plan_info& info, int64_t n_samp, size_t bytes,
               RingLayout* L) {
  for (int n = 2; n <= kRingMaxSegments; ++n) {
    if (!ring_layout(p, info, n_samp, n, L)) return false;
    if (L->bytes() <= bytes) return true;
  }
  return false;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" {

const char* dd_status_string(dd_status status) {
  switch (status) {
    case DD_OK: return "DD_OK";
    case DD_ERR_INVALID_ARG: return "DD_ERR_INVALID_ARG";
    case DD_ERR_UNSUPPORTED: return "DD_ERR_UNSUPPORTED";
    case DD_ERR_SHAPE: return "DD_ERR_SHAPE";
    case DD_ERR_BUDGET: return "DD_ERR_BUDGET";
    case DD_ERR_CUDA: return "DD_ERR_CUDA";
    case DD_ERR_TIMEOUT: return "DD_ERR_TIMEOUT";
  }
  return "DD_ERR_UNKNOWN";
}

const char* dd_last_error_detail(void) { return g_detail.c_str(); }

const char* dd_version(void) { return "gb300-dedisp 0.1 (sm_103a)"; }

dd_status dd_plan_create(const double* freqs_mhz, int32_t n_chan, double f_ref_mhz,
                         double t_samp_s, const dd_range* ranges, int32_t n_ranges,
                         dd_dtype dtype, dd_plan* out) {
  g_detail.clear();
  if (!out) return fail(DD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!freqs_mhz || !ranges) return fail(DD_ERR_INVALID_ARG, "freqs or ranges is NULL");
  if (n_chan <= 0 || n_chan > (1 << 20)) return fail(DD_ERR_INVALID_ARG, "n_chan out of range");
  if (n_ranges <= 0 || n_ranges > DD_MAX_RANGES)
    return fail(DD_ERR_INVALID_ARG, "n_ranges must be in [1, DD_MAX_RANGES]");
  if (dtype != DD_U8 && dtype != DD_U16 && dtype != DD_F32 && dtype != DD_U4)
    return fail(DD_ERR_INVALID_ARG, "unknown dtype");
  if (!(t_samp_s > 0.0) || !std::isfinite(t_samp_s)) return fail(DD_ERR_INVALID_ARG, "t_samp must be > 0");
  if (!(f_ref_mhz > 0.0) || !std::isfinite(f_ref_mhz)) return fail(DD_ERR_INVALID_ARG, "f_ref must be > 0");
  for (int32_t c = 0; c < n_chan; ++c) {
    if (!(freqs_mhz[c] > 0.0) || !(freqs_mhz[c] <= f_ref_mhz))
      return fail(DD_ERR_INVALID_ARG, "channel frequency outside (0, f_ref]");
  }
  for (int32_t i = 0; i < n_ranges; ++i) {
    const dd_range& r = ranges[i];
    if (!(r.dm_step > 0.0) || !(r.dm_hi > r.dm_lo) || !(r.dm_lo >= 0.0) || r.bin < 1 ||
        r.bin > 1024 || !std::isfinite(r.dm_hi))
      return fail(DD_ERR_INVALID_ARG, "range needs step > 0, hi > lo >= 0, 1 <= bin <= 1024");
  }
  dd_plan_s* p = new (std::nothrow) dd_plan_s();
  if (!p) return fail(DD_ERR_INVALID_ARG, "host allocation failed");
  p->n_chan = n_chan;
  p->f_ref = f_ref_mhz;
  p->t_samp = t_samp_s;
  p->dtype = dtype;
  p->freqs.assign(freqs_mhz, freqs_mhz + n_chan);
  p->ranges.resize(n_ranges);
  for (int32_t i = 0; i < n_ranges; ++i) p->ranges[i].r = ranges[i];
  dd_status st;
  try {
    st = build_plan(p);
  } catch (const std::bad_alloc&) {
    st = fail(DD_ERR_INVALID_ARG, "host allocation failed while planning");
  }
  if (st != DD_OK) {
    delete p;
    return st;
  }
  *out = p;
  return DD_OK;
}

dd_status dd_plan_destroy(dd_plan plan) {
  if (plan) free_host_pipe(plan);
  delete plan;
  return DD_OK;
}

dd_status dd_plan_query(dd_plan plan, int64_t n_samp, dd_plan_info* out) {
  if (!plan || !out) return fail(DD_ERR_INVALID_ARG, "plan or out is NULL");
  if (n_samp < 0) return fail(DD_ERR_INVALID_ARG, "n_samp < 0");
  return fill_info(plan, n_samp, out);
}

dd_status dd_plan_shifts(dd_plan plan, int32_t range, int32_t* host_out) {
  if (!plan || !host_out) return fail(DD_ERR_INVALID_ARG, "plan or host_out is NULL");
  if (range < 0 || range >= static_cast<int32_t>(plan->ranges.size()))
    return fail(DD_ERR_INVALID_ARG, "range index out of bounds");
  const auto& s = plan->ranges[range].shifts;
  std::memcpy(host_out, s.data(), s.size() * sizeof(int32_t));
  return DD_OK;
}

dd_status dd_plan_dm_ranges(const double* freqs_mhz, int32_t n_chan, double t_samp_s,
                            double dm_max, double tol, double width_s, int32_t max_bin,
                            int32_t max_ranges, dd_range* out, int32_t* n_ranges) {
  if (!freqs_mhz || !out || !n_ranges) return fail(DD_ERR_INVALID_ARG, "NULL argument");
  if (n_chan < 2 || !(tol > 1.0) || !(dm_max > 0.0) || !(t_samp_s > 0.0) || !(width_s >= 0.0) ||
      max_bin < 1 || max_ranges < 1)
    return fail(DD_ERR_INVALID_ARG, "need n_chan >= 2, tol > 1, dm_max > 0, t_samp > 0, "
                                    "width >= 0, max_bin >= 1, max_ranges >= 1");
  for (int32_t c = 0; c < n_chan; ++c)
    if (!(freqs_mhz[c] > 0.0)) return fail(DD_ERR_INVALID_ARG, "frequencies must be positive");
  double f_lo = freqs_mhz[0], f_hi = freqs_mhz[0];
  for (int32_t c = 1; c < n_chan; ++c) {
    f_lo = std::min(f_lo, freqs_mhz[c]);
    f_hi = std::max(f_hi, freqs_mhz[c]);
  }
  if (!(f_hi > f_lo)) return fail(DD_ERR_INVALID_ARG, "the band has no width");
  *n_ranges = dm_plan_ranges(freqs_mhz, n_chan, t_samp_s, dm_max, tol, width_s, max_bin,
                             std::min(max_ranges, DD_MAX_RANGES), out);
  return DD_OK;
}

dd_status dd_plan_set_tile(dd_plan plan, int32_t range, int32_t tile) {
  if (!plan) return fail(DD_ERR_INVALID_ARG, "plan is NULL");
  if (range < 0 || range >= static_cast<int32_t>(plan->ranges.size()))
    return fail(DD_ERR_INVALID_ARG, "range index out of bounds");
  if (tile != 0 && tile != DD_TILE_PATTERN && tile != DD_TILE_PACKED && !tk::shape_for(tile))
    return fail(DD_ERR_INVALID_ARG, "tile must be 0, 1, 2, 4, 6, 8, DD_TILE_PATTERN or DD_TILE_PACKED");
  bool ok;
  try {
    ok = retile_range(plan, static_cast<size_t>(range), tile, -1);
  } catch (const std::bad_alloc&) {
    return fail(DD_ERR_INVALID_ARG, "host allocation failed while retiling");
  }
  // A refused tile leaves the previous tables (rebuilt identically) and the
  // workspace binding as they were; a new tile needs dd_plan_upload.
  if (!ok) return fail(DD_ERR_UNSUPPORTED, "tile cannot serve this range");
  plan->d_ws = nullptr;
  return DD_OK;
}

dd_status dd_tile_shapes(dd_tile_shape* out, int32_t max_shapes, int32_t* n_shapes) {
  if (!n_shapes || (max_shapes > 0 && !out)) return fail(DD_ERR_INVALID_ARG, "NULL argument");
  const int32_t n = tk::kNumPatShapes;
  *n_shapes = n;
  for (int32_t i = 0; i < n && i < max_shapes; ++i) {
    const tk::PatShape& s = tk::kPatShapes[i];
    out[i].words_per_lane = s.h;
    out[i].dms_per_lane = tk::kPatDr;
    out[i].warps = s.warps;
    out[i].channels_per_stage = s.nc;
    out[i].channel_pairs = s.pairs ? 1 : 0;
    out[i].float_pairs = s.h < 15 ? 1 : 0;
    out[i].automatic = i < tk::kPatTuneFirst ? 1 : 0;
  }
  return DD_OK;
}

dd_status dd_plan_set_tile_shape(dd_plan plan, int32_t range, int32_t tile, int32_t shape) {
  if (!plan) return fail(DD_ERR_INVALID_ARG, "plan is NULL");
  if (range < 0 || range >= static_cast<int32_t>(plan->ranges.size()))
    return fail(DD_ERR_INVALID_ARG, "range index out of bounds");
  if (tile != DD_TILE_PATTERN && tile != DD_TILE_PACKED)
    return fail(DD_ERR_INVALID_ARG, "tile must be DD_TILE_PATTERN or DD_TILE_PACKED");
  if (shape < -1 || shape >= tk::kNumPatShapes)
    return fail(DD_ERR_INVALID_ARG, "shape must be -1 or a dd_tile_shapes index");
  bool ok;
  try {
    ok = retile_range(plan, static_cast<size_t>(range), tile, shape);
  } catch (const std::bad_alloc&) {
    return fail(DD_ERR_INVALID_ARG, "host allocation failed while retiling");
  }
  if (!ok) return fail(DD_ERR_UNSUPPORTED, "that shape cannot serve this range");
  plan->d_ws = nullptr;
  return DD_OK;
}

dd_status dd_plan_set_wait_limit(dd_plan plan, int32_t max_polls, int32_t hold_stage) {
  if (!plan) return fail(DD_ERR_INVALID_ARG, "plan is NULL");
  if (hold_stage < -1) return fail(DD_ERR_INVALID_ARG, "hold_stage must be -1 or a stage index");
  plan->wait_iters = max_polls > 0 ? max_polls : tk::kWaitIters;
  plan->hold_stage = hold_stage;
  return DD_OK;
}

dd_status dd_plan_upload(dd_plan plan, void* d_workspace, size_t bytes, void* stream) {
  if (!plan || !d_workspace) return fail(DD_ERR_INVALID_ARG, "plan or workspace is NULL");
  if (bytes < plan->ws_bytes) return fail(DD_ERR_BUDGET, "workspace smaller than workspace_bytes");
  if (!aligned16(d_workspace)) return fail(DD_ERR_SHAPE, "workspace must be 16-byte aligned");
  // The image ends before the widening slots, which need no contents.
  cudaError_t e = cudaMemcpyAsync(d_workspace, plan->host_ws.data(), plan->host_ws.size(),
                                  cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "dd_plan_upload");
  plan->d_ws = d_workspace;
  return DD_OK;
}

static dd_status check_run(dd_plan plan, const void* d_in, int64_t stride, int64_t n_samp,
                           const void* d_out, dd_plan_info* info) {
  if (!plan || !d_in || !d_out) return fail(DD_ERR_INVALID_ARG, "plan, d_in or d_out is NULL");
  if (!plan->d_ws) return fail(DD_ERR_INVALID_ARG, "plan has no uploaded workspace");
  if (n_samp <= 0 || stride < n_samp) return fail(DD_ERR_SHAPE, "need 0 < n_samp <= row stride");
  if (!aligned16(d_in) || !aligned16(d_out)) return fail(DD_ERR_SHAPE, "d_in/d_out must be 16-byte aligned");
  if (plan->dtype == DD_U4 ? stride % 32 != 0
                            : (stride * static_cast<int64_t>(elem_size(plan->dtype))) % 16 != 0)
    return fail(DD_ERR_SHAPE, "row stride must be a multiple of 16 bytes");
  fill_info(plan, n_samp, info);
  for (int32_t i = 0; i < info->n_ranges; ++i)
    if (info->n_out[i] <= 0) return fail(DD_ERR_SHAPE, "input shorter than a range's maximum delay");
  return DD_OK;
}

// The ring: the ranges with a copy kind run in time segments from a ring of
// kRingSlots packed slots.  Segment k is packed (on the plan's high-priority
// packing stream) into slot k % kRingSlots once the kernels of segment
// k - kRingSlots have read it, and its kernels run on the caller's stream
// (k even) or the plan's second compute stream (k odd), so that packing
// overlaps the kernels and one segment's last CTAs overlap the next one's
// first.  The other ranges read the input on the caller's stream.  The
// caller's stream waits for all of it.
static dd_status run_ring(dd_plan plan, const dd_plan_info& info, const void* d_in,
                          int64_t in_row_stride, int64_t n_samp, void* d_out, void* d_scratch,
                          const RingLayout& L, void* stream) {
  std::lock_guard<std::mutex> lock(g_pipe_mu);
  HostPipe* hp = nullptr;
  cudaError_t e = host_pipe(plan, &hp);
  if (e != cudaSuccess) return cuda_fail(e, "dd_run ring streams");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  e = cudaEventRecord(hp->start, s);
  for (cudaStream_t o : {hp->s_pack, hp->s_comp})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(o, hp->start, 0);
  if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run ring ordering");
  unsigned char* out = static_cast<unsigned char*>(d_out);
  for (size_t r = 0; r < plan->ranges.size(); ++r) {
    if (L.ring[r]) continue;
    const int le = launch_range(plan, plan->ranges[r], d_in, in_row_stride, n_samp, info.n_out[r],
                                out + info.out_offset[r] * 4, 0, info.n_out[r], s);
    if (le != 0) return fail_joined(hp, s, le, "dd_run forward launch");
  }
  const size_t in_bytes = dtype_row_bytes(plan->dtype, in_row_stride);
  for (size_t k = 0; k < L.segs.size(); ++k) {
    const RingSeg& sg = L.segs[k];
    const int slot = static_cast<int>(k % kRingSlots);
    unsigned char* buf = static_cast<unsigned char*>(d_scratch) + slot * L.slot_bytes;
    if (k >= static_cast<size_t>(kRingSlots)) {
      e = cudaStreamWaitEvent(hp->s_pack, hp->freed[slot], 0);
      if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run ring ordering");
    }
    int le = launch_pack_pairs(d_in, static_cast<int64_t>(in_bytes), plan->n_chan, n_samp, buf,
                               L.slot_words, L.pair, sg.origin, sg.end,
                               pack_source(plan->dtype), hp->s_pack, sg.origin);
    if (le != 0) return fail_joined(hp, s, le, "dd_run ring packing");
    cudaStream_t sc = (k & 1) ? hp->s_comp : s;
    e = cudaEventRecord(hp->packed[slot], hp->s_pack);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, hp->packed[slot], 0);
    if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run ring ordering");
    for (size_t r = 0; r < plan->ranges.size(); ++r) {
      if (!L.ring[r] || sg.hi[r] <= sg.lo[r]) continue;
      const RangePlan& rp = plan->ranges[r];
      le = launch_range(plan, rp, buf, L.slot_words, n_samp, info.n_out[r],
                        out + info.out_offset[r] * 4, sg.lo[r], sg.hi[r], sc,
                        copy_kind(rp, true), sg.origin);
      if (le != 0) return fail_joined(hp, s, le, "dd_run ring forward launch");
    }
    e = cudaEventRecord(hp->freed[slot], sc);
    if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run ring ordering");
  }
  e = cudaEventRecord(hp->done, hp->s_comp);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hp->done, 0);
  if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run ring ordering");
  return DD_OK;
}

// The forward transform of every range.  n_keep == nullptr: all n_out_r
// outputs of each range, at dd_plan_query's offsets.  Otherwise the first
// n_keep[r] outputs of range r, as rows of n_keep[r] samples, concatenated.
// pack == false: the packed copy is already in d_scratch (dd_pack_input).
// Scratch that holds the full copies of every range with a copy kind runs
// them all from packed copies; less scratch runs them from the ring when it
// fits (whole outputs, packing here); else only the DD_TILE_PACKED ranges
// read packed copies.
static dd_status run_forward(dd_plan plan, const void* d_in, int64_t in_row_stride,
                             int64_t n_samp, const int64_t* n_keep, void* d_out, void* d_scratch,
                             size_t scratch_bytes, void* stream, bool pack = true) {
  dd_plan_info info;
  dd_status st = check_run(plan, d_in, in_row_stride, n_samp, d_out, &info);
  if (st != DD_OK) return st;
  if (n_keep) {
    for (int32_t i = 0; i < info.n_ranges; ++i)
      if (n_keep[i] < 1 || n_keep[i] > info.n_out[i])
        return fail(DD_ERR_SHAPE, "n_keep[r] must be in [1, n_out_r]");
  }
  if (d_scratch && reinterpret_cast<uintptr_t>(d_scratch) % 16 != 0)
    return fail(DD_ERR_SHAPE, "input scratch must be 16-byte aligned");
  const bool with_auto = full_with_auto(plan, n_samp, d_scratch, scratch_bytes);
  if (!n_keep && pack && d_scratch && scratch_bytes < packed_input_bytes(plan, n_samp, true)) {
    RingLayout L;
    if (pick_ring(plan, info, n_samp, scratch_bytes, &L))
      return run_ring(plan, info, d_in, in_row_stride, n_samp, d_out, d_scratch, L, stream);
  }
  const size_t need = packed_input_bytes(plan, n_samp, with_auto);
  if (need > 0) {
    if (!d_scratch)
      return fail(DD_ERR_UNSUPPORTED,
                  "a range is on DD_TILE_PACKED: run it with dd_run_scratch and scratch of "
                  "dd_plan_input_scratch_bytes");
    if (scratch_bytes < need) return fail(DD_ERR_BUDGET, "input scratch too small");
    if (reinterpret_cast<uintptr_t>(d_scratch) % 16 != 0)
      return fail(DD_ERR_SHAPE, "input scratch must be 16-byte aligned");
  }
  std::vector<int32_t> range_copy;
  const std::vector<PackedCopy> copies = packed_copies(plan, n_samp, &range_copy, with_auto);
  if (pack)
    for (const PackedCopy& pc : copies) {
      const int e = launch_pack_copy(plan, pc, d_in, in_row_stride, n_samp, d_scratch, stream);
      if (e != 0) return cuda_fail(e, "dd_run packing");
    }
  const size_t osz = 4;
  int64_t off = 0;           // element offset of the range's rows in d_out
  for (size_t i = 0; i < plan->ranges.size(); ++i) {
    const RangePlan& rp = plan->ranges[i];
    const int64_t row = n_keep ? n_keep[i] : info.n_out[i];
    void* o = static_cast<unsigned char*>(d_out) + (n_keep ? off : info.out_offset[i]) * osz;
    off += rp.n_dm * row;
    const void* src = d_in;
    int64_t stride = in_row_stride;
    int kind = 0;
    if (range_copy[i] >= 0) {  // reads its packed copy
      const PackedCopy& pc = copies[range_copy[i]];
      src = static_cast<unsigned char*>(d_scratch) + pc.offset;
      stride = pc.stride;
      kind = copy_kind(rp, with_auto);
    }
    int e = launch_range(plan, rp, src, stride, n_samp, row, o, 0, row, stream, kind);
    if (e != 0) return cuda_fail(e, "dd_run forward launch");
  }
  return DD_OK;
}

dd_status dd_run_scratch(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                         void* d_out, void* d_scratch, size_t scratch_bytes, void* stream) {
  return run_forward(plan, d_in, in_row_stride, n_samp, nullptr, d_out, d_scratch, scratch_bytes,
                     stream);
}

dd_status dd_pack_input(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                        void* d_scratch, size_t scratch_bytes, void* stream) {
  dd_plan_info info;
  if (!d_scratch) return fail(DD_ERR_INVALID_ARG, "d_scratch is NULL");
  dd_status st = check_run(plan, d_in, in_row_stride, n_samp, d_scratch, &info);
  if (st != DD_OK) return st;
  const bool with_auto = full_with_auto(plan, n_samp, d_scratch, scratch_bytes);
  const size_t need = packed_input_bytes(plan, n_samp, with_auto);
  if (need == 0) return DD_OK;  // no range reads a packed copy
  if (scratch_bytes < need) return fail(DD_ERR_BUDGET, "input scratch too small");
  if (reinterpret_cast<uintptr_t>(d_scratch) % 16 != 0)
    return fail(DD_ERR_SHAPE, "input scratch must be 16-byte aligned");
  for (const PackedCopy& pc : packed_copies(plan, n_samp, nullptr, with_auto)) {
    const int e = launch_pack_copy(plan, pc, d_in, in_row_stride, n_samp, d_scratch, stream);
    if (e != 0) return cuda_fail(e, "dd_pack_input");
  }
  return DD_OK;
}

dd_status dd_run_packed(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                        void* d_out, const void* d_scratch, size_t scratch_bytes, void* stream) {
  return run_forward(plan, d_in, in_row_stride, n_samp, nullptr, d_out,
                     const_cast<void*>(d_scratch), scratch_bytes, stream, false);
}

dd_status dd_run_window(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                        const int64_t* n_keep, void* d_out, void* d_scratch, size_t scratch_bytes,
                        void* stream) {
  if (!n_keep) return fail(DD_ERR_INVALID_ARG, "n_keep is NULL");
  return run_forward(plan, d_in, in_row_stride, n_samp, n_keep, d_out, d_scratch, scratch_bytes,
                     stream);
}

dd_status dd_run(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                 void* d_out, void* stream) {
  return dd_run_scratch(plan, d_in, in_row_stride, n_samp, d_out, nullptr, 0, stream);
}

dd_status dd_plan_input_scratch_bytes(dd_plan plan, int64_t n_samp, size_t* bytes) {
  if (!plan || !bytes) return fail(DD_ERR_INVALID_ARG, "plan or bytes is NULL");
  if (n_samp <= 0) return fail(DD_ERR_SHAPE, "n_samp must be positive");
  *bytes = packed_input_bytes(plan, n_samp);
  return DD_OK;
}

dd_status dd_plan_packed_scratch_bytes(dd_plan plan, int64_t n_samp, int32_t n_segments,
                                       size_t* bytes) {
  if (!plan || !bytes) return fail(DD_ERR_INVALID_ARG, "plan or bytes is NULL");
  if (n_samp <= 0) return fail(DD_ERR_SHAPE, "n_samp must be positive");
  if (n_segments < 1 || n_segments > kRingMaxSegments)
    return fail(DD_ERR_INVALID_ARG, "n_segments must be in [1, 256]");
  *bytes = 0;
  const size_t full = packed_input_bytes(plan, n_samp, true);
  if (full == 0 || n_segments == 1) {
    *bytes = full;
    return DD_OK;
  }
  dd_plan_info info;
  fill_info(plan, n_samp, &info);
  for (int32_t i = 0; i < info.n_ranges; ++i)
    if (info.n_out[i] <= 0) return fail(DD_ERR_SHAPE, "input shorter than a range's maximum delay");
  RingLayout L;
  if (!ring_layout(plan, info, n_samp, n_segments, &L))
    return fail(DD_ERR_UNSUPPORTED,
                "the packed ranges need copies at a bin above 1 or at two pair distances: "
                "no ring (n_segments = 1 gives the full copies)");
  // At least the full copies' size, the run takes those instead.
  *bytes = L.bytes();
  return DD_OK;
}

dd_status dd_run_adjoint_scratch(dd_plan plan, const float* d_ybar, float* d_xbar,
                                 int64_t n_samp, int64_t xbar_row_stride, void* d_scratch,
                                 size_t scratch_bytes, void* stream) {
  if (plan && plan->dtype != DD_F32) return fail(DD_ERR_UNSUPPORTED, "adjoint needs a float32 plan");
  if (d_scratch && reinterpret_cast<uintptr_t>(d_scratch) % 16 != 0)
    return fail(DD_ERR_SHAPE, "adjoint scratch must be 16-byte aligned");
  dd_plan_info info;
  dd_status st = check_run(plan, d_ybar, xbar_row_stride, n_samp, d_xbar, &info);
  if (st != DD_OK) return st;
  int e = launch_adjoint(plan, d_ybar, d_xbar, n_samp, xbar_row_stride, info.n_out,
                         info.out_offset, d_scratch, scratch_bytes, stream);
  if (e != 0) return cuda_fail(e, "dd_run_adjoint launch");
  return DD_OK;
}

dd_status dd_run_adjoint(dd_plan plan, const float* d_ybar, float* d_xbar, int64_t n_samp,
                         int64_t xbar_row_stride, void* stream) {
  return dd_run_adjoint_scratch(plan, d_ybar, d_xbar, n_samp, xbar_row_stride, nullptr, 0,
                                stream);
}

dd_status dd_adjoint_scratch_bytes(dd_plan plan, int64_t n_samp, size_t* bytes) {
  if (!plan || !bytes) return fail(DD_ERR_INVALID_ARG, "plan or bytes is NULL");
  if (plan->dtype != DD_F32) return fail(DD_ERR_UNSUPPORTED, "adjoint needs a float32 plan");
  if (n_samp <= 0) return fail(DD_ERR_SHAPE, "n_samp must be positive");
  *bytes = adjoint_scratch_bytes(plan, n_samp);
  return DD_OK;
}

dd_status dd_plan_device_status(dd_plan plan, void* stream) {
  if (!plan || !plan->d_ws) return fail(DD_ERR_INVALID_ARG, "plan has no uploaded workspace");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, plan->d_ws, sizeof(word), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "dd_plan_device_status");
  if (word != 0) {
    const int32_t zero = 0;
    e = cudaMemcpyAsync(plan->d_ws, &zero, sizeof(zero), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "dd_plan_device_status reset");
    return fail(DD_ERR_TIMEOUT, "a bounded device wait gave up during an earlier run");
  }
  return DD_OK;
}

// The segmented host pipeline of dd_run_host (tm == nullptr: h_in is
// channel-major with row stride cm_stride, copied straight into d_cm) and
// dd_run_host_tmajor (h_in is time-major with row stride tm_stride, copied
// into d_tm and transposed into d_cm on its own stream).  With d_packed
// (ranges on DD_TILE_PACKED, channel-major input only), the packed copy of
// each segment's columns is made on that stream too, `pair` samples behind the
// copied ones (a packed word needs samples t and t + pair), and those ranges'
// kernels take only outputs whose words are packed.
static dd_status run_host_pipeline(dd_plan plan, const dd_plan_info& info, const void* h_in,
                                   int64_t tm_stride, void* d_tm, int64_t n_samp, void* h_out,
                                   void* d_cm, int64_t cm_stride, void* d_out_stage,
                                   void* d_packed, bool with_auto, void* stream) {
  std::lock_guard<std::mutex> lock(g_pipe_mu);
  HostPipe* hp = nullptr;
  cudaError_t e = host_pipe(plan, &hp);
  if (e != cudaSuccess) return cuda_fail(e, "dd_run_host streams");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t esz = elem_size(plan->dtype);
  const bool tmajor = d_tm != nullptr;
  const unsigned char* hin = static_cast<const unsigned char*>(h_in);
  unsigned char* dtm = static_cast<unsigned char*>(d_tm);
  unsigned char* dcm = static_cast<unsigned char*>(d_cm);
  unsigned char* hout = static_cast<unsigned char*>(h_out);
  unsigned char* dout = static_cast<unsigned char*>(d_out_stage);
  // The other streams start after the caller's earlier work on `stream`.
  e = cudaEventRecord(hp->start, s);
  for (cudaStream_t o : {hp->s_in, hp->s_out, hp->s_comp, hp->s_tr})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(o, hp->start, 0);
  if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
  const int64_t seg = (n_samp + kHostSegments - 1) / kHostSegments;
  const int64_t seg_len = (seg + 255) / 256 * 256;
  const int64_t packed_stride = (n_samp + 3) / 4 * 4;
  int32_t pair = -1;  // lag of the packed copy behind the copied samples (-1: none)
  for (const auto& rp : plan->ranges)
    if (d_packed && copy_kind(rp, with_auto)) pair = pack_pair(rp, copy_kind(rp, with_auto));
  int64_t packed_done = 0;
  int64_t raw_done = 0;
  int64_t done[DD_MAX_RANGES] = {};
  for (int k = 0; k < kHostSegments; ++k) {
    const bool last = k == kHostSegments - 1;
    cudaStream_t sc = (k & 1) ? hp->s_comp : s;
    const int64_t raw_end = last ? n_samp : std::min<int64_t>(n_samp, (k + 1) * seg_len);
    // Segment k of the raw samples, every channel.
    cudaEvent_t ready = hp->in[k];
    if (raw_end > raw_done) {
      if (tmajor) {  // whole time rows: one contiguous block
        const size_t pitch = static_cast<size_t>(tm_stride) * esz;
        e = cudaMemcpyAsync(dtm + raw_done * pitch, hin + raw_done * pitch,
                            static_cast<size_t>(raw_end - raw_done) * pitch,
                            cudaMemcpyHostToDevice, hp->s_in);
      } else {       // a column block of every channel row (a strided 2-D copy)
        const size_t pitch = row_bytes(plan->dtype, cm_stride);
        const size_t b0 = row_bytes(plan->dtype, raw_done);  // raw_done is even
        e = cudaMemcpy2DAsync(dcm + b0, pitch, hin + b0, pitch,
                              row_bytes(plan->dtype, raw_end) - b0, plan->n_chan,
                              cudaMemcpyHostToDevice, hp->s_in);
      }
      if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host input copy");
    }
    e = cudaEventRecord(hp->in[k], hp->s_in);
    if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
    if (tmajor) {  // transposes run in order on one stream
      e = cudaStreamWaitEvent(hp->s_tr, hp->in[k], 0);
      if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
      if (raw_end > raw_done) {
        const int le = launch_transpose(static_cast<int>(esz), dtm, tm_stride, plan->n_chan, dcm,
                                        cm_stride, raw_done, raw_end, hp->s_tr);
        if (le != 0) return fail_joined(hp, s, le, "dd_run_host transpose");
      }
      e = cudaEventRecord(hp->tr[k], hp->s_tr);
      if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
      ready = hp->tr[k];
    } else if (pair >= 0) {  // packed copy of the columns whose pair partner is in
      e = cudaStreamWaitEvent(hp->s_tr, hp->in[k], 0);
      if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
      const int64_t packed_end =
          last ? packed_stride : std::max(packed_done, (raw_end - pair) / 16 * 16);
      if (packed_end > packed_done) {
        const int le = launch_pack_pairs(dcm, row_bytes(plan->dtype, cm_stride), plan->n_chan,
                                         n_samp, d_packed, packed_stride, pair, packed_done,
                                         packed_end, pack_source(plan->dtype), hp->s_tr);
        if (le != 0) return fail_joined(hp, s, le, "dd_run_host packing");
      }
      packed_done = packed_end;
      e = cudaEventRecord(hp->tr[k], hp->s_tr);
      if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
      ready = hp->tr[k];
    }
    raw_done = std::max(raw_done, raw_end);
    e = cudaStreamWaitEvent(sc, ready, 0);
    if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
    // Every output whose dispersion track ends inside the samples copied so
    // far: t + S_max < raw_end / bin, whole time tiles except at the end.
    int64_t lim[DD_MAX_RANGES];
    for (size_t r = 0; r < plan->ranges.size(); ++r) {
      const RangePlan& rp = plan->ranges[r];
      const int kind = pair >= 0 ? copy_kind(rp, with_auto) : 0;
      const bool from_packed = kind != 0;
      const int64_t n_out = info.n_out[r];
      int64_t l = n_out;
      if (!last) {
        // Samples usable so far; a packed word t holds samples t and t + pair.
        const int64_t avail = from_packed ? packed_done + pair : raw_end;
        const int64_t ts = range_tile_samples(rp);
        l = std::min<int64_t>(n_out, avail / rp.r.bin - rp.s_max);
        l = l < 0 ? 0 : l / ts * ts;
      }
      lim[r] = l;
      if (l > done[r]) {
        const int le = launch_range(plan, rp, from_packed ? d_packed : dcm,
                                    from_packed ? packed_stride : cm_stride, n_samp, n_out,
                                    dout + info.out_offset[r] * 4, done[r], l, sc, kind);
        if (le != 0) return fail_joined(hp, s, le, "dd_run_host forward launch");
      }
    }
    e = cudaEventRecord(hp->comp[k], sc);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->s_out, hp->comp[k], 0);
    if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
    for (size_t r = 0; r < plan->ranges.size(); ++r) {
      if (lim[r] <= done[r]) continue;
      const size_t pitch_out = static_cast<size_t>(info.n_out[r]) * 4;
      const size_t off = static_cast<size_t>(info.out_offset[r] + done[r]) * 4;
      e = cudaMemcpy2DAsync(hout + off, pitch_out, dout + off, pitch_out,
                            static_cast<size_t>(lim[r] - done[r]) * 4,
                            static_cast<size_t>(info.n_dm[r]), cudaMemcpyDeviceToHost,
                            hp->s_out);
      if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host output copy");
      done[r] = lim[r];
    }
  }
  // The caller's stream completes after the last output copy, which follows
  // every segment's kernels on both compute streams.
  e = cudaEventRecord(hp->done, hp->s_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hp->done, 0);
  if (e != cudaSuccess) return fail_joined(hp, s, e, "dd_run_host ordering");
  return DD_OK;
}

dd_status dd_run_host_scratch(dd_plan plan, const void* h_in, int64_t in_row_stride,
                              int64_t n_samp, void* h_out, void* d_in_stage, void* d_out_stage,
                              void* d_scratch, size_t scratch_bytes, void* stream) {
  if (!h_in || !h_out) return fail(DD_ERR_INVALID_ARG, "h_in or h_out is NULL");
  dd_plan_info info;
  dd_status st = check_run(plan, d_in_stage, in_row_stride, n_samp, d_out_stage, &info);
  if (st != DD_OK) return st;
  // Automatic tiles with a copy kind read the packed copy too when the
  // scratch holds it and it is the one bin-1 copy the pipeline makes.
  bool with_auto = full_with_auto(plan, n_samp, d_scratch, scratch_bytes);
  if (with_auto) {
    const auto all = packed_copies(plan, n_samp, nullptr, true);
    with_auto = all.size() == 1 && all[0].bin == 1;
  }
  const size_t need = packed_input_bytes(plan, n_samp, with_auto);
  if (need > 0) {
    if (!d_scratch)
      return fail(DD_ERR_UNSUPPORTED,
                  "a range is on DD_TILE_PACKED: run it with dd_run_host_scratch and scratch of "
                  "dd_plan_input_scratch_bytes");
    if (scratch_bytes < need) return fail(DD_ERR_BUDGET, "input scratch too small");
    if (reinterpret_cast<uintptr_t>(d_scratch) % 16 != 0)
      return fail(DD_ERR_SHAPE, "input scratch must be 16-byte aligned");
    const auto copies = packed_copies(plan, n_samp, nullptr, with_auto);
    if (copies.size() != 1 || copies[0].bin != 1)
      return fail(DD_ERR_UNSUPPORTED,
                  "the host pipeline packs one copy at bin 1: binned packed ranges run "
                  "through dd_run_scratch");
  }
  return run_host_pipeline(plan, info, h_in, 0, nullptr, n_samp, h_out, d_in_stage,
                           in_row_stride, d_out_stage, need > 0 ? d_scratch : nullptr,
                           with_auto, stream);
}

dd_status dd_run_host(dd_plan plan, const void* h_in, int64_t in_row_stride, int64_t n_samp,
                      void* h_out, void* d_in_stage, void* d_out_stage, void* stream) {
  return dd_run_host_scratch(plan, h_in, in_row_stride, n_samp, h_out, d_in_stage, d_out_stage,
                             nullptr, 0, stream);
}

static dd_status check_transpose(size_t esz, const void* d_in, int64_t in_row_stride,
                                 int32_t n_chan, const void* d_out, int64_t out_row_stride,
                                 int64_t t_begin, int64_t t_end) {
  if (!d_in || !d_out) return fail(DD_ERR_INVALID_ARG, "d_in or d_out is NULL");
  if (n_chan <= 0 || in_row_stride < n_chan || t_begin < 0 || t_end < t_begin ||
      t_end > out_row_stride)
    return fail(DD_ERR_SHAPE, "need n_chan <= in_row_stride and 0 <= t_begin <= t_end <= "
                              "out_row_stride");
  if (!aligned16(d_in) || !aligned16(d_out) ||
      (in_row_stride * static_cast<int64_t>(esz)) % 16 != 0 ||
      (out_row_stride * static_cast<int64_t>(esz)) % 16 != 0)
    return fail(DD_ERR_SHAPE, "buffers and row strides must be 16-byte aligned");
  if (t_begin % static_cast<int64_t>(4 / esz) != 0)
    return fail(DD_ERR_SHAPE, "t_begin must be a multiple of 4 / sample bytes");
  return DD_OK;
}

dd_status dd_transpose(dd_dtype dtype, const void* d_in, int64_t in_row_stride, int32_t n_chan,
                       void* d_out, int64_t out_row_stride, int64_t t_begin, int64_t t_end,
                       void* stream) {
  if (dtype != DD_U8 && dtype != DD_U16 && dtype != DD_F32)
    return fail(dtype == DD_U4 ? DD_ERR_UNSUPPORTED : DD_ERR_INVALID_ARG,
                "dd_transpose takes uint8, uint16 or float32 samples");
  const size_t esz = elem_size(dtype);
  dd_status st = check_transpose(esz, d_in, in_row_stride, n_chan, d_out, out_row_stride,
                                 t_begin, t_end);
  if (st != DD_OK) return st;
  const int e = launch_transpose(static_cast<int>(esz), d_in, in_row_stride, n_chan, d_out,
                                 out_row_stride, t_begin, t_end, stream);
  if (e != 0) return cuda_fail(e, "dd_transpose launch");
  return DD_OK;
}

dd_status dd_run_host_tmajor(dd_plan plan, const void* h_in, int64_t in_row_stride,
                             int64_t n_samp, void* h_out, void* d_tm_stage, void* d_cm_stage,
                             int64_t cm_row_stride, void* d_out_stage, void* stream) {
  if (!h_in || !h_out || !d_tm_stage) return fail(DD_ERR_INVALID_ARG, "NULL buffer");
  if (plan && packed_input_bytes(plan, 1) > 0)
    return fail(DD_ERR_UNSUPPORTED, "the host pipeline does not take DD_TILE_PACKED ranges");
  if (plan && plan->dtype == DD_U4)
    return fail(DD_ERR_UNSUPPORTED, "time-major input takes uint8, uint16 or float32 samples");
  dd_plan_info info;
  dd_status st = check_run(plan, d_cm_stage, cm_row_stride, n_samp, d_out_stage, &info);
  if (st != DD_OK) return st;
  st = check_transpose(elem_size(plan->dtype), d_tm_stage, in_row_stride, plan->n_chan,
                       d_cm_stage, cm_row_stride, 0, n_samp);
  if (st != DD_OK) return st;
  return run_host_pipeline(plan, info, h_in, in_row_stride, d_tm_stage, n_samp, h_out,
                           d_cm_stage, cm_row_stride, d_out_stage, nullptr, false, stream);
}

}  // extern "C"
