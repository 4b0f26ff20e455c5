// batch.cu -- C ABI of the persistent batch runtime (include/dd.h, dd_batch_*).
//
// Many beams -- plans of different channel counts, dtypes, sampling times and
// DM plans -- are dedispersed by persistent launches whose CTAs take (job, DM
// block, time tile) items from a device counter until the list is exhausted:
// one launch of the pattern-tile kernel (fwd_pattern_batch.cu) for the ranges
// on pattern tiles and one of the offset-tile kernel (fwd_tiled.cu) for the
// others (the two register footprints differ: 16 warps x 128 registers
// against 12 x 168).  Items are ordered longest first (largest channel count
// x tile work), DM blocks of a time tile consecutive so their shared input
// window stays in L2.  dd_batch_bind uploads the per-job pointers once;
// dd_batch_run is then a counter reset and up to two launches, which a CUDA
// graph can capture and replay.  The launches run on lanes: one per pattern
// group and one for the offset family, each lane a stream (the first the
// caller's) that packs its beams' inputs and then runs its persistent launch,
// so packing overlaps other lanes' compute and the lanes' tails overlap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dd_internal.h"
#include "fwd_tiled.h"

struct dd_batch_s {
  std::vector<dd_plan> plans;
  std::vector<int64_t> n_samp;
  struct JobRef {
    int32_t plan;
    int32_t range;
    int64_t n_out;
    int64_t out_offset;  // elements into the plan's output
    bool pattern;        // on a pattern tile (else an offset tile)
    int32_t index;       // job number within its family
  };
  std::vector<JobRef> jobs;
  std::vector<dd::tk::BatchItem> items;    // offset-tile family
  std::vector<dd::tk::BatchJob> host_jobs;
  std::vector<dd::tk::PatBatchJob> host_pjobs;
  // Pattern-tile jobs grouped by variant (kind, shape): one launch each.
  struct PatGroup {
    int32_t kind;
    int32_t shape;
    int mode = 0;  // widening mode every job takes (tk::widen_mode; set when bound)
    size_t smem = 0;
    size_t off_items = 0;
    std::vector<dd::tk::BatchItem> items;
  };
  std::vector<PatGroup> groups;
  std::vector<int32_t> pjob_group;  // group of each pattern job
  int32_t max_lraw = 0;
  int32_t max_lp = 0;
  size_t off_jobs = 0, off_items = 0, off_pjobs = 0, ws_bytes = 0;
  unsigned char* d_ws = nullptr;
  bool bound = false;
  int32_t sm_count = 0;
  // Plans with ranges on DD_TILE_PACKED: the packing pass each run makes
  // before the persistent launches (bound by dd_batch_bind_scratch).
  struct Pack {
    int32_t plan;
    dd::PackedCopy copy{};  // one packed copy of the plan's input (api.cu)
    int32_t copy_index = 0;
    const void* in = nullptr;
    int64_t in_stride = 0;  // samples
    void* scratch = nullptr;
    int32_t lane = 0;       // launch lane that packs it (the first lane reading it)
  };
  std::vector<Pack> packs;
  // Launch lanes: one per pattern group, then the offset-tile family.  Each
  // lane runs its packing launches and then its persistent launch on a stream
  // of its own (the first lane on the caller's), so that packing overlaps the
  // other lanes' compute and one lane's tail overlaps the next lane's start.
  std::vector<std::vector<int32_t>> lane_packs;  // packs each lane reads
  std::vector<cudaStream_t> lane_streams;        // [n_lanes]; [0] unused (caller's)
  std::vector<cudaEvent_t> pack_done, lane_done;
  cudaEvent_t start = nullptr;
  ~dd_batch_s() {
    for (cudaStream_t st : lane_streams)
      if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : pack_done)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : lane_done)
      if (e) cudaEventDestroy(e);
    if (start) cudaEventDestroy(start);
  }
};

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

bool batch_shape(int32_t dr) {
  for (int d : dd::tk::kBatchDr)
    if (d == dr && dd::tk::shape_for(dr)->warps == dd::tk::kBatchWarps) return true;
  return false;
}

}  // namespace

using namespace dd;

extern "C" {

dd_status dd_batch_create(const dd_plan* plans, const int64_t* n_samp, int32_t n_plans,
                          dd_batch* out) {
  if (!out) return fail(DD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!plans || !n_samp || n_plans <= 0) return fail(DD_ERR_INVALID_ARG, "no plans");
  dd_batch_s* b = new (std::nothrow) dd_batch_s();
  if (!b) return fail(DD_ERR_INVALID_ARG, "host allocation failed");
  try {
    struct Cost {
      double per_item;
      int32_t job;
    };
    std::vector<Cost> order;
    for (int32_t i = 0; i < n_plans; ++i) {
      const dd_plan p = plans[i];
      if (!p) {
        delete b;
        return fail(DD_ERR_INVALID_ARG, "NULL plan in batch");
      }
      b->plans.push_back(p);
      b->n_samp.push_back(n_samp[i]);
      int64_t out_off = 0;
      for (size_t r = 0; r < p->ranges.size(); ++r) {
        const RangePlan& rp = p->ranges[r];
        const bool pat = rp.tile_ok && rp.tile_pattern;
        if (r == 0) {  // the plan's packed copies (one per distinct pair distance and bin)
          const auto copies = packed_copies(p, n_samp[i], nullptr);
          for (size_t k = 0; k < copies.size(); ++k) {
            dd_batch_s::Pack pk{i};
            pk.copy = copies[k];
            pk.copy_index = static_cast<int32_t>(k);
            b->packs.push_back(pk);
          }
        }
        if (!rp.tile_ok || (rp.tile_pattern && !pat) ||
            (!pat && (rp.tile_pattern || !batch_shape(rp.tile_dr)))) {
          delete b;
          return fail(DD_ERR_UNSUPPORTED,
                      "batch plan " + std::to_string(i) + " range " + std::to_string(r) +
                          " is not on a batch tile (the pattern or packed tile, or the offset "
                          "tile with 4/2/1 DMs per lane; see dd_plan_set_tile)");
        }
        const int64_t n_out = range_n_out(p, rp, n_samp[i]);
        if (n_out <= 0) {
          delete b;
          return fail(DD_ERR_SHAPE, "batch plan " + std::to_string(i) + " input too short");
        }
        const int32_t job = static_cast<int32_t>(b->jobs.size());
        int32_t index;
        int ts;
        double dms;
        if (pat) {
          const tk::PatShape& ps = tk::kPatShapes[rp.tile_shape];
          index = static_cast<int32_t>(b->host_pjobs.size());
          b->host_pjobs.emplace_back();
          size_t g = 0;
          while (g < b->groups.size() &&
                 !(b->groups[g].kind == rp.tile_kind && b->groups[g].shape == rp.tile_shape))
            ++g;
          if (g == b->groups.size()) b->groups.push_back({rp.tile_kind, rp.tile_shape});
          b->pjob_group.push_back(static_cast<int32_t>(g));
          b->groups[g].smem = std::max(
              b->groups[g].smem,
              tk::pat_smem_bytes(rp.tile_kind, tk::staged_bin(rp.tile_kind, rp.r.bin), ps,
                                 rp.tile_lp));
          ts = tk::pat_tile_samples(rp.tile_kind, ps.h);
          dms = static_cast<double>(ps.warps) * tk::kPatDr;
        } else {
          index = static_cast<int32_t>(b->host_jobs.size());
          b->host_jobs.emplace_back();
          b->max_lraw = std::max(b->max_lraw, tk::raw_bytes(rp.tile_kind, rp.r.bin, rp.tile_lp));
          b->max_lp = std::max(b->max_lp, rp.tile_lp);
          ts = tk::tile_samples(rp.tile_kind);
          dms = static_cast<double>(tk::shape_for(rp.tile_dr)->warps) * rp.tile_dr;
        }
        b->jobs.push_back({i, static_cast<int32_t>(r), n_out, out_off, pat, index});
        out_off += rp.n_dm * n_out;
        order.push_back({static_cast<double>(p->n_chan) * dms * ts * rp.r.bin, job});
      }
    }
    // Longest items first; within a job, DM blocks of a time tile together.
    std::stable_sort(order.begin(), order.end(),
                     [](const Cost& a, const Cost& c) { return a.per_item > c.per_item; });
    for (const Cost& c : order) {
      const auto& j = b->jobs[c.job];
      const dd_plan p = b->plans[j.plan];
      const RangePlan& rp = p->ranges[j.range];
      const int ts = j.pattern ? tk::pat_tile_samples(rp.tile_kind, rp.tile_h)
                               : tk::tile_samples(rp.tile_kind);
      const int64_t tiles = (j.n_out + ts - 1) / ts;
      auto& list = j.pattern ? b->groups[b->pjob_group[j.index]].items : b->items;
      for (int64_t t = 0; t < tiles; ++t)
        for (int32_t blk = 0; blk < rp.tile_n_blocks; ++blk)
          list.push_back({j.index, blk, static_cast<int32_t>(t), 0});
    }
    size_t n_pitems = 0;
    for (const auto& g : b->groups) n_pitems += g.items.size();
    if (b->items.size() > 0x7fffffffu || n_pitems > 0x7fffffffu ||
        b->groups.size() + 1 > tk::kStatusBytes / sizeof(uint32_t)) {
      delete b;
      return fail(DD_ERR_BUDGET, "too many batch items");
    }
    size_t ws = tk::kStatusBytes;  // work counters of the two launches
    ws = align256(ws);
    b->off_jobs = ws;
    ws += b->host_jobs.size() * sizeof(tk::BatchJob);
    ws = align256(ws);
    b->off_pjobs = ws;
    ws += b->host_pjobs.size() * sizeof(tk::PatBatchJob);
    ws = align256(ws);
    b->off_items = ws;
    ws += b->items.size() * sizeof(tk::BatchItem);
    for (auto& g : b->groups) {
      ws = align256(ws);
      g.off_items = ws;
      ws += g.items.size() * sizeof(tk::BatchItem);
    }
    b->ws_bytes = align256(ws);
    const size_t smem = tk::batch_smem_bytes(b->max_lraw, b->max_lp);
    bool too_big = !b->items.empty() && smem > 227 * 1024;
    for (const auto& g : b->groups) too_big = too_big || g.smem > 227 * 1024;
    if (too_big) {
      delete b;
      return fail(DD_ERR_BUDGET, "batch shared-memory layout exceeds 227 KB");
    }
    // Lanes that read each plan's packed copy (offset tiles never do).
    b->lane_packs.assign(b->groups.size() + 1, {});
    for (size_t k = 0; k < b->packs.size(); ++k) {
      int32_t first = -1;
      std::vector<int32_t> range_copy;
      packed_copies(b->plans[b->packs[k].plan], b->n_samp[b->packs[k].plan], &range_copy);
      for (const auto& j : b->jobs) {
        if (j.plan != b->packs[k].plan || !j.pattern) continue;
        if (range_copy[j.range] != b->packs[k].copy_index) continue;
        const int32_t lane = b->pjob_group[j.index];
        auto& lp = b->lane_packs[lane];
        if (std::find(lp.begin(), lp.end(), static_cast<int32_t>(k)) == lp.end())
          lp.push_back(static_cast<int32_t>(k));
        if (first < 0) first = lane;
      }
      b->packs[k].lane = first < 0 ? 0 : first;
    }
  } catch (const std::bad_alloc&) {
    delete b;
    return fail(DD_ERR_INVALID_ARG, "host allocation failed while building the batch");
  }
  *out = b;
  return DD_OK;
}

dd_status dd_batch_destroy(dd_batch batch) {
  delete batch;
  return DD_OK;
}

dd_status dd_batch_workspace_bytes(dd_batch batch, size_t* bytes) {
  if (!batch || !bytes) return fail(DD_ERR_INVALID_ARG, "batch or bytes is NULL");
  *bytes = batch->ws_bytes;
  return DD_OK;
}

dd_status dd_batch_info(dd_batch batch, int64_t* n_items, int32_t* n_jobs) {
  if (!batch || !n_items || !n_jobs) return fail(DD_ERR_INVALID_ARG, "NULL argument");
  int64_t n = static_cast<int64_t>(batch->items.size());
  for (const auto& g : batch->groups) n += static_cast<int64_t>(g.items.size());
  *n_items = n;
  *n_jobs = static_cast<int32_t>(batch->jobs.size());
  return DD_OK;
}

dd_status dd_batch_launches(dd_batch batch, int32_t* n_launches) {
  if (!batch || !n_launches) return fail(DD_ERR_INVALID_ARG, "NULL argument");
  int32_t n = (batch->items.empty() ? 0 : 1) + static_cast<int32_t>(batch->packs.size());
  for (const auto& g : batch->groups) n += g.items.empty() ? 0 : 1;
  *n_launches = n;
  return DD_OK;
}

dd_status dd_batch_upload(dd_batch batch, void* d_workspace, size_t bytes, void* stream) {
  if (!batch || !d_workspace) return fail(DD_ERR_INVALID_ARG, "batch or workspace is NULL");
  if (bytes < batch->ws_bytes) return fail(DD_ERR_BUDGET, "workspace smaller than needed");
  if (reinterpret_cast<uintptr_t>(d_workspace) & 255u)
    return fail(DD_ERR_SHAPE, "batch workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(d_workspace);
  cudaError_t e = cudaSuccess;
  if (!batch->items.empty())
    e = cudaMemcpyAsync(ws + batch->off_items, batch->items.data(),
                        batch->items.size() * sizeof(tk::BatchItem), cudaMemcpyHostToDevice, s);
  for (const auto& g : batch->groups)
    if (e == cudaSuccess && !g.items.empty())
      e = cudaMemcpyAsync(ws + g.off_items, g.items.data(), g.items.size() * sizeof(tk::BatchItem),
                          cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "dd_batch_upload");
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "dd_batch_upload device query");
  batch->sm_count = sms;
  batch->d_ws = ws;
  batch->bound = false;
  if (batch->lane_streams.empty()) {  // the launch lanes' streams and events (dd_batch_run)
    const size_t n_lanes = batch->groups.size() + 1;
    batch->lane_streams.assign(n_lanes, nullptr);
    batch->lane_done.assign(n_lanes, nullptr);
    batch->pack_done.assign(batch->packs.size(), nullptr);
    for (size_t i = 1; i < n_lanes && e == cudaSuccess; ++i)
      e = cudaStreamCreateWithFlags(&batch->lane_streams[i], cudaStreamNonBlocking);
    for (size_t i = 0; i < n_lanes && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&batch->lane_done[i], cudaEventDisableTiming);
    for (size_t i = 0; i < batch->packs.size() && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&batch->pack_done[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&batch->start, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "dd_batch_upload streams");
  }
  return DD_OK;
}

dd_status dd_batch_plan_scratch_bytes(dd_batch batch, int32_t plan, size_t* bytes) {
  if (!batch || !bytes) return fail(DD_ERR_INVALID_ARG, "batch or bytes is NULL");
  if (plan < 0 || plan >= static_cast<int32_t>(batch->plans.size()))
    return fail(DD_ERR_INVALID_ARG, "plan index out of bounds");
  return dd_plan_input_scratch_bytes(batch->plans[plan], batch->n_samp[plan], bytes);
}

dd_status dd_batch_bind_scratch(dd_batch batch, const void* const* d_in,
                                const int64_t* in_row_stride, void* const* d_out,
                                void* const* d_scratch, const size_t* scratch_bytes,
                                void* stream) {
  if (!batch || !d_in || !in_row_stride || !d_out)
    return fail(DD_ERR_INVALID_ARG, "NULL argument");
  if (!batch->d_ws) return fail(DD_ERR_INVALID_ARG, "batch has no uploaded workspace");
  batch->bound = false;
  for (auto& pk : batch->packs) {
    const dd_plan p = batch->plans[pk.plan];
    size_t need = 0;
    dd_plan_input_scratch_bytes(p, batch->n_samp[pk.plan], &need);
    if (!d_scratch || !scratch_bytes || !d_scratch[pk.plan])
      return fail(DD_ERR_UNSUPPORTED, "batch plan " + std::to_string(pk.plan) +
                                          " has a packed-tile range: bind it with scratch");
    if (scratch_bytes[pk.plan] < need) return fail(DD_ERR_BUDGET, "batch plan scratch too small");
    if (reinterpret_cast<uintptr_t>(d_scratch[pk.plan]) & 15u)
      return fail(DD_ERR_SHAPE, "batch plan scratch must be 16-byte aligned");
    pk.in = d_in[pk.plan];
    pk.in_stride = in_row_stride[pk.plan];
    pk.scratch = d_scratch[pk.plan];
  }
  for (auto& g : batch->groups) g.mode = -1;  // none seen yet
  for (size_t j = 0; j < batch->jobs.size(); ++j) {
    const auto& jr = batch->jobs[j];
    const dd_plan p = batch->plans[jr.plan];
    if (!p->d_ws) return fail(DD_ERR_INVALID_ARG, "a batch plan has no uploaded workspace");
    const void* x = d_in[jr.plan];
    void* o = d_out[jr.plan];
    int64_t stride = in_row_stride[jr.plan];
    const int64_t n = batch->n_samp[jr.plan];
    const int64_t stride_bytes = p->dtype == DD_U4 ? stride / 2
                                 : stride * (p->dtype == DD_U8 ? 1 : (p->dtype == DD_U16 ? 2 : 4));
    if (!x || !o) return fail(DD_ERR_INVALID_ARG, "NULL input or output pointer");
    if ((reinterpret_cast<uintptr_t>(x) & 15u) || (reinterpret_cast<uintptr_t>(o) & 15u) ||
        stride < n || stride_bytes % 16 != 0 || (p->dtype == DD_U4 && stride % 2 != 0))
      return fail(DD_ERR_SHAPE, "batch input/output alignment or stride");
    const RangePlan& rp = p->ranges[jr.range];
    if (rp.tile_ok && tk::packed_copy_kind(rp.tile_kind)) {  // reads its packed copy
      std::vector<int32_t> range_copy;
      const auto copies = packed_copies(p, n, &range_copy);
      const PackedCopy& pc = copies[range_copy[jr.range]];
      x = static_cast<unsigned char*>(d_scratch[jr.plan]) + pc.offset;
      stride = pc.stride;
    }
    const tk::TileParams prm =
        tiled_params(p, rp, static_cast<unsigned char*>(p->d_ws) + rp.off_tile_recs,
                     reinterpret_cast<int32_t*>(static_cast<unsigned char*>(p->d_ws) +
                                                tk::kStatusOffset),
                     x, stride, jr.n_out, static_cast<char*>(o) + jr.out_offset * 4);
    if (jr.pattern) {
      tk::PatBatchJob& bj = batch->host_pjobs[jr.index];
      auto& grp = batch->groups[batch->pjob_group[jr.index]];
      const int m = tk::widen_mode(rp.tile_kind, tk::kPatShapes[rp.tile_shape].nc,
                                   prm.wslots != nullptr, prm.flush);
      // A group whose jobs would take different modes widens into the rows.
      grp.mode = grp.mode < 0 || grp.mode == m ? m : 0;
      bj.p = prm;
      bj.kind = rp.tile_kind;
      bj.shape = rp.tile_shape;
    } else {
      tk::BatchJob& bj = batch->host_jobs[jr.index];
      bj.p = prm;
      bj.kind = rp.tile_kind;
      bj.dr = rp.tile_dr;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!batch->host_jobs.empty())
    e = cudaMemcpyAsync(batch->d_ws + batch->off_jobs, batch->host_jobs.data(),
                        batch->host_jobs.size() * sizeof(tk::BatchJob), cudaMemcpyHostToDevice,
                        s);
  if (e == cudaSuccess && !batch->host_pjobs.empty())
    e = cudaMemcpyAsync(batch->d_ws + batch->off_pjobs, batch->host_pjobs.data(),
                        batch->host_pjobs.size() * sizeof(tk::PatBatchJob),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "dd_batch_bind");
  batch->bound = true;
  return DD_OK;
}

dd_status dd_batch_bind(dd_batch batch, const void* const* d_in, const int64_t* in_row_stride,
                        void* const* d_out, void* stream) {
  return dd_batch_bind_scratch(batch, d_in, in_row_stride, d_out, nullptr, nullptr, stream);
}

dd_status dd_batch_run(dd_batch batch, void* stream) {
  if (!batch) return fail(DD_ERR_INVALID_ARG, "batch is NULL");
  if (!batch->bound) return fail(DD_ERR_INVALID_ARG, "batch is not bound (dd_batch_bind)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e =
      cudaMemsetAsync(batch->d_ws, 0, (1 + batch->groups.size()) * sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "dd_batch_run counter reset");
  // Lanes: pattern groups 0..G-1, then the offset family (lane G).  Lane 0
  // runs on the caller's stream, the others on the batch's own streams, which
  // start after the counter reset and end before the caller's stream goes on.
  const size_t n_lanes = batch->groups.size() + 1;
  std::vector<bool> used(n_lanes, false);
  for (size_t gi = 0; gi < batch->groups.size(); ++gi) used[gi] = !batch->groups[gi].items.empty();
  used[n_lanes - 1] = !batch->items.empty();
  if (batch->lane_streams.size() != n_lanes) return fail(DD_ERR_INVALID_ARG, "batch not uploaded");
  auto lane_stream = [&](size_t lane) {
    return lane == 0 ? s : batch->lane_streams[lane];
  };
  e = cudaEventRecord(batch->start, s);
  for (size_t i = 1; i < n_lanes && e == cudaSuccess; ++i)
    if (used[i]) e = cudaStreamWaitEvent(batch->lane_streams[i], batch->start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "dd_batch_run ordering");
  // Packing launches, each on the first lane that reads its copy.
  for (size_t k = 0; k < batch->packs.size(); ++k) {
    const auto& pk = batch->packs[k];
    cudaStream_t ls = lane_stream(pk.lane);
    const int le = launch_pack_copy(batch->plans[pk.plan], pk.copy, pk.in, pk.in_stride,
                                    batch->n_samp[pk.plan], pk.scratch, ls);
    if (le != 0) return cuda_fail(le, "dd_batch_run packing");
    e = cudaEventRecord(batch->pack_done[k], ls);
    if (e != cudaSuccess) return cuda_fail(e, "dd_batch_run ordering");
  }
  for (size_t gi = 0; gi < batch->groups.size(); ++gi) {
    const auto& g = batch->groups[gi];
    if (g.items.empty()) continue;
    cudaStream_t ls = lane_stream(gi);
    for (int32_t k : batch->lane_packs[gi])  // copies packed on another lane
      if (batch->packs[k].lane != static_cast<int32_t>(gi)) {
        e = cudaStreamWaitEvent(ls, batch->pack_done[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "dd_batch_run ordering");
      }
    tk::PatBatchArgs args{};
    args.jobs = reinterpret_cast<const tk::PatBatchJob*>(batch->d_ws + batch->off_pjobs);
    args.items = reinterpret_cast<const tk::BatchItem*>(batch->d_ws + g.off_items);
    args.n_items = static_cast<int32_t>(g.items.size());
    args.counter = reinterpret_cast<uint32_t*>(batch->d_ws) + 1 + gi;
    const int64_t grid = std::min<int64_t>(static_cast<int64_t>(g.items.size()),
                                           static_cast<int64_t>(batch->sm_count));
    int le = launch_pattern_batch(g.kind, g.shape, args,
                                  static_cast<int32_t>(std::max<int64_t>(grid, 1)), g.smem, ls,
                                  g.mode < 0 ? 0 : g.mode);
    if (le != 0) return cuda_fail(le, "dd_batch_run pattern launch");
  }
  if (!batch->items.empty()) {
    cudaStream_t ls = lane_stream(n_lanes - 1);
    tk::BatchArgs args{};
    args.jobs = reinterpret_cast<const tk::BatchJob*>(batch->d_ws + batch->off_jobs);
    args.items = reinterpret_cast<const tk::BatchItem*>(batch->d_ws + batch->off_items);
    args.n_items = static_cast<int32_t>(batch->items.size());
    args.counter = reinterpret_cast<uint32_t*>(batch->d_ws);
    args.max_lraw = batch->max_lraw;
    const size_t smem = tk::batch_smem_bytes(batch->max_lraw, batch->max_lp);
    const int64_t grid = std::min<int64_t>(static_cast<int64_t>(batch->items.size()),
                                           static_cast<int64_t>(batch->sm_count));
    int le = launch_batch(args, static_cast<int32_t>(std::max<int64_t>(grid, 1)), smem, ls);
    if (le != 0) return cuda_fail(le, "dd_batch_run launch");
  }
  // The caller's stream goes on once every lane is done (packs only run on
  // lanes with items: the lanes that read them).
  for (size_t i = 1; i < n_lanes; ++i) {
    if (!used[i]) continue;
    e = cudaEventRecord(batch->lane_done[i], batch->lane_streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, batch->lane_done[i], 0);
    if (e != cudaSuccess) return cuda_fail(e, "dd_batch_run ordering");
  }
  return DD_OK;
}

dd_status dd_batch_status(dd_batch batch, void* stream) {
  if (!batch) return fail(DD_ERR_INVALID_ARG, "batch is NULL");
  dd_status worst = DD_OK;
  for (const dd_plan p : batch->plans) {
    dd_status st = dd_plan_device_status(p, stream);
    if (st != DD_OK) worst = st;
  }
  return worst;
}

}  // extern "C"
