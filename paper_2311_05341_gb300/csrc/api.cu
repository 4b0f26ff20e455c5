// api.cu -- the C ABI of libdd (declared in include/dd.h): argument checking,
// error reporting and kernel dispatch.  No device memory is allocated here.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "dd_internal.h"

namespace dd {

namespace {
thread_local std::string g_detail;
}

dd_status fail(dd_status st, const std::string& detail) {
  g_detail = detail;
  return st;
}

dd_status cuda_fail(int err, const char* what) {
  g_detail = std::string(what) + ": " + cudaGetErrorName(static_cast<cudaError_t>(err)) +
             " (" + cudaGetErrorString(static_cast<cudaError_t>(err)) + ")";
  return DD_ERR_CUDA;
}

namespace {

size_t elem_size(dd_dtype t) { return t == DD_U8 ? 1 : (t == DD_U16 ? 2 : 4); }

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
    o->tile_dms[i] = !rp.tile_ok ? 0 : (rp.tile_pattern ? DD_TILE_PATTERN : rp.tile_dr);
    int64_t raw = (static_cast<int64_t>(rp.s_max) + 1) * rp.r.bin - 1;
    if (raw > o->max_delay_raw) o->max_delay_raw = raw;
  }
  o->out_elems = off;
  o->workspace_bytes = p->ws_bytes;
  return DD_OK;
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
  if (dtype != DD_U8 && dtype != DD_U16 && dtype != DD_F32)
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

dd_status dd_plan_set_tile(dd_plan plan, int32_t range, int32_t tile) {
  if (!plan) return fail(DD_ERR_INVALID_ARG, "plan is NULL");
  if (range < 0 || range >= static_cast<int32_t>(plan->ranges.size()))
    return fail(DD_ERR_INVALID_ARG, "range index out of bounds");
  if (tile != 0 && tile != DD_TILE_PATTERN && !tk::shape_for(tile))
    return fail(DD_ERR_INVALID_ARG, "tile must be 0, 1, 2, 4, 6, 8 or DD_TILE_PATTERN");
  bool ok;
  try {
    ok = retile_range(plan, static_cast<size_t>(range), tile);
  } catch (const std::bad_alloc&) {
    return fail(DD_ERR_INVALID_ARG, "host allocation failed while retiling");
  }
  plan->d_ws = nullptr;  // tables changed: upload again
  if (!ok) return fail(DD_ERR_UNSUPPORTED, "tile cannot serve this range");
  return DD_OK;
}

dd_status dd_plan_upload(dd_plan plan, void* d_workspace, size_t bytes, void* stream) {
  if (!plan || !d_workspace) return fail(DD_ERR_INVALID_ARG, "plan or workspace is NULL");
  if (bytes < plan->ws_bytes) return fail(DD_ERR_BUDGET, "workspace smaller than workspace_bytes");
  if (!aligned16(d_workspace)) return fail(DD_ERR_SHAPE, "workspace must be 16-byte aligned");
  cudaError_t e = cudaMemcpyAsync(d_workspace, plan->host_ws.data(), plan->ws_bytes,
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
  if ((stride * static_cast<int64_t>(elem_size(plan->dtype))) % 16 != 0)
    return fail(DD_ERR_SHAPE, "row stride must be a multiple of 16 bytes");
  fill_info(plan, n_samp, info);
  for (int32_t i = 0; i < info->n_ranges; ++i)
    if (info->n_out[i] <= 0) return fail(DD_ERR_SHAPE, "input shorter than a range's maximum delay");
  return DD_OK;
}

dd_status dd_run(dd_plan plan, const void* d_in, int64_t in_row_stride, int64_t n_samp,
                 void* d_out, void* stream) {
  dd_plan_info info;
  dd_status st = check_run(plan, d_in, in_row_stride, n_samp, d_out, &info);
  if (st != DD_OK) return st;
  const size_t osz = 4;
  for (size_t i = 0; i < plan->ranges.size(); ++i) {
    void* o = static_cast<unsigned char*>(d_out) + info.out_offset[i] * osz;
    const RangePlan& rp = plan->ranges[i];
    int e = rp.tile_ok ? launch_forward_tiled(plan, rp, d_in, in_row_stride, n_samp,
                                              info.n_out[i], o, stream)
                       : launch_forward_generic(plan, rp, d_in, in_row_stride, n_samp,
                                                info.n_out[i], o, stream);
    if (e != 0) return cuda_fail(e, "dd_run forward launch");
  }
  return DD_OK;
}

dd_status dd_run_adjoint(dd_plan plan, const float* d_ybar, float* d_xbar, int64_t n_samp,
                         int64_t xbar_row_stride, void* stream) {
  if (plan && plan->dtype != DD_F32) return fail(DD_ERR_UNSUPPORTED, "adjoint needs a float32 plan");
  dd_plan_info info;
  dd_status st = check_run(plan, d_ybar, xbar_row_stride, n_samp, d_xbar, &info);
  if (st != DD_OK) return st;
  int e = launch_adjoint(plan, d_ybar, d_xbar, n_samp, xbar_row_stride, info.n_out,
                         info.out_offset, stream);
  if (e != 0) return cuda_fail(e, "dd_run_adjoint launch");
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

dd_status dd_run_host(dd_plan plan, const void* h_in, int64_t in_row_stride, int64_t n_samp,
                      void* h_out, void* d_in_stage, void* d_out_stage, void* stream) {
  if (!h_in || !h_out) return fail(DD_ERR_INVALID_ARG, "h_in or h_out is NULL");
  dd_plan_info info;
  dd_status st = check_run(plan, d_in_stage, in_row_stride, n_samp, d_out_stage, &info);
  if (st != DD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t in_bytes = static_cast<size_t>(plan->n_chan) * in_row_stride * elem_size(plan->dtype);
  cudaError_t e = cudaMemcpyAsync(d_in_stage, h_in, in_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "dd_run_host input copy");
  st = dd_run(plan, d_in_stage, in_row_stride, n_samp, d_out_stage, stream);
  if (st != DD_OK) return st;
  e = cudaMemcpyAsync(h_out, d_out_stage, static_cast<size_t>(info.out_elems) * 4,
                      cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "dd_run_host output copy");
  return DD_OK;
}

}  // extern "C"
