// static_scratch.cu -- dd_run_u8_noalloc: the uint8 tiled forward transform for
// callers that cannot allocate device memory.
//
// dd_run needs a caller-allocated workspace holding the plan's tables.  Some
// callers cannot provide one: a real-time pipeline that must not call
// cudaMalloc while observing (it can synchronise the device and stall the
// data stream), a plug-in whose host framework owns every device allocation,
// or a process running under a fixed memory budget that is already spent.
// This entry point keeps the tables in a fixed-size array in the library's own
// device memory instead (file-scope __device__ storage, reserved on every GPU
// that loads the library until the process exits) and allocates nothing.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "dd_internal.h"
#include "fwd_tiled.h"

namespace dd {
namespace {

// Status word (tk::kStatusBytes) followed by each range's record table.
constexpr size_t kStaticScratchBytes = size_t{8} << 20;  // 8 MiB
static_assert(kStaticScratchBytes % 256 == 0, "scratch size must keep 256-byte alignment");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
// Device address of the array per device, looked up once with that device
// current and kept for the life of the process (a cudaDeviceReset between
// calls would leave it stale; that is documented as unsupported).
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Device address of the scratch array on the current device (set-up once per
// device, with that device current).
dd_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "dd_run_u8_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(DD_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "dd_run_u8_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return DD_OK;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" dd_status dd_run_u8_noalloc(dd_plan plan, const void* d_in, int64_t in_row_stride,
                                       int64_t n_samp, void* d_out, void* stream) {
  if (!plan || !d_in || !d_out) return fail(DD_ERR_INVALID_ARG, "plan, d_in or d_out is NULL");
  if (plan->dtype != DD_U8) return fail(DD_ERR_UNSUPPORTED, "dd_run_u8_noalloc needs a uint8 plan");
  if (n_samp <= 0 || in_row_stride < n_samp)
    return fail(DD_ERR_SHAPE, "need 0 < n_samp <= row stride");
  if ((reinterpret_cast<uintptr_t>(d_in) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 15u))
    return fail(DD_ERR_SHAPE, "d_in/d_out must be 16-byte aligned");
  if (in_row_stride % 16 != 0) return fail(DD_ERR_SHAPE, "row stride must be a multiple of 16 bytes");

  // Every range must run on the tiled kernel, and all tables must fit.
  size_t need = tk::kStatusBytes;
  for (const RangePlan& rp : plan->ranges) {
    if (!rp.tile_ok || tk::packed_copy_kind(rp.tile_kind))
      return fail(DD_ERR_UNSUPPORTED,
                  "dd_run_u8_noalloc needs every range on the tiled kernel, not DD_TILE_PACKED");
    if (range_n_out(plan, rp, n_samp) <= 0)
      return fail(DD_ERR_SHAPE, "input shorter than a range's maximum delay");
    need = align256(need) + rp.tile_recs.size();
  }
  if (align256(need) > kStaticScratchBytes)
    return fail(DD_ERR_BUDGET, "plan tables need " + std::to_string(align256(need)) +
                                   " bytes; dd_run_u8_noalloc holds at most " +
                                   std::to_string(kStaticScratchBytes));

  unsigned char* scratch = nullptr;
  dd_status st = scratch_for_current_device(&scratch);
  if (st != DD_OK) return st;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The status word is zero when the library loads; kernels only set bits in
  // it and dd_run_u8_noalloc_status clears it, so it collects every call's
  // timeouts until it is read.
  int32_t* err = reinterpret_cast<int32_t*>(scratch + tk::kStatusOffset);
  cudaError_t e = cudaSuccess;
  size_t off = tk::kStatusBytes;
  int64_t out_off = 0;
  for (const RangePlan& rp : plan->ranges) {
    off = align256(off);
    e = cudaMemcpyAsync(scratch + off, rp.tile_recs.data(), rp.tile_recs.size(),
                        cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "dd_run_u8_noalloc: copy tables");
    const int64_t n_out = range_n_out(plan, rp, n_samp);
    int32_t* o = static_cast<int32_t*>(d_out) + out_off;
    int le = launch_forward_tiled_with_tables(plan, rp, scratch + off, err, d_in, in_row_stride,
                                              n_out, o, 0, n_out, stream, false);
    if (le != 0) return cuda_fail(le, "dd_run_u8_noalloc launch");
    off += rp.tile_recs.size();
    out_off += rp.n_dm * n_out;
  }
  return DD_OK;
}

extern "C" dd_status dd_run_u8_noalloc_status(void* stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "dd_run_u8_noalloc_status: cudaGetDevice");
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (dev >= 0 && dev < kMaxDevices) scratch = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  if (!scratch) return DD_OK;  // no call has run on this device
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t word = 0;
  e = cudaMemcpyAsync(&word, scratch + tk::kStatusOffset, sizeof(word), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "dd_run_u8_noalloc_status: read status");
  if (word == 0) return DD_OK;
  e = cudaMemsetAsync(scratch + tk::kStatusOffset, 0, sizeof(word), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "dd_run_u8_noalloc_status: clear status");
  return fail(DD_ERR_TIMEOUT, "a bounded device wait of an earlier dd_run_u8_noalloc call gave up");
}
