// fwd_u8.cu -- register-tiled uint8 dedispersion kernel for sm_103a.
//
// Computes Eq. 3 (Algorithm 1) for 8-bit input at time bin 1:
//     Y[d][t] = sum_c X[c][t + s(c, d)]
// exactly (integer sums), with the same output partition as the paper's GPU
// kernel (Sec. 4: a CTA owns D_dm x D_t outputs, threads keep accumulators in
// registers, Algorithm 3) but organised for GB300's issue rate:
//
//  * CTA = 8 warps x 32 lanes.  The CTA owns 64 consecutive DMs and 1280 output
//    samples.  Warp w owns DMs d0 + 8w .. d0 + 8w + 7; every lane owns the same
//    8 DMs x 40 samples.
//  * Samples are summed two per 32-bit word in 16-bit lanes (SIMD within a
//    word, Sec. 4.1): word u of a channel's staged window packs samples u and
//    u + 640 (the pairing distance is half the CTA tile, so lane l's 20 words
//    cover samples [20l, 20l + 20) and [640 + 20l, 640 + 20l + 20)).  One
//    2-input add adds two samples; 255 * 256 < 2^16, so the lanes are widened
//    (flushed) to int32 every 256 channels.
//  * Staging (Algorithm 3's B_loc): per channel, the raw bytes of the window
//    starting at t0 + s(c, d0) are fetched with one TMA bulk copy
//    (cp.async.bulk, 16-byte aligned, completion on an mbarrier), two stages
//    in flight; all threads then re-pack them into paired 16-bit words.
//  * Register reuse across DMs: each lane loads its 36-word window of a
//    channel once (9 x 16-byte shared loads) and adds it into all 8 DMs.  The
//    offset of DM i inside the window is a per-(channel, warp) 4-bit value
//    (the paper's T_diff * Delta t_pc of Eq. 6, resolved to an integer on the
//    host); a warp-uniform switch selects the register slice, so the adds use
//    compile-time register indices.
//  * The widen/flush goes through shared memory (transposed, conflict-free) and
//    adds into the int32 output rows with coalesced loads and stores.
//
// Every wait on an mbarrier is bounded; on timeout the kernel records
// DD_ERR_TIMEOUT in the plan's device status word and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"
#include "fwd_u8.h"

namespace dd {
namespace u8k {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Bounded wait for phase `parity` of an mbarrier.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kWaitIters; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  return __byte_perm(a, b, sel);
}

struct Smem {
  uint32_t bar_base;   // 2 mbarriers
  Rec* recs;           // [2][kNC]
  uint8_t* raw;        // [2][kNC][lraw]
  uint32_t* pw;        // [kNC][lp]
};

// Issue the TMA copies of stage `st` into buffer `buf`.  Threads 0..kNC-1 copy
// one channel each, thread kNC copies the stage's records.
__device__ __forceinline__ void issue_stage(const U8Params& p, const Smem& sm, int st, int buf,
                                            int64_t t0, int32_t base, int tid) {
  const uint32_t bar = sm.bar_base + 8u * buf;
  const int c0 = st * kNC;
  if (tid < kNC) {
    const int c = c0 + tid;
    uint32_t bytes = 0;
    const uint8_t* src = nullptr;
    if (c < p.n_chan) {
      const int64_t ua = (t0 + base) & ~int64_t(15);
      if (ua < p.stride) {
        const int64_t room = p.stride - ua;
        bytes = static_cast<uint32_t>(room < p.lraw ? room : p.lraw);
        src = p.x + static_cast<int64_t>(c) * p.stride + ua;
      }
    }
    mbar_arrive_expect(bar, bytes);
    if (bytes) {
      uint8_t* dst = sm.raw + (static_cast<size_t>(buf) * kNC + tid) * p.lraw;
      bulk_copy(smem_u32(dst), src, bytes, bar);
    }
  } else if (tid == kNC) {
    const int nc = min(kNC, p.n_chan - c0);
    const uint32_t bytes = static_cast<uint32_t>(nc) * sizeof(Rec);
    mbar_arrive_expect(bar, bytes);
    const Rec* src = p.recs + static_cast<int64_t>(blockIdx.x % p.n_blocks) * p.n_chan + c0;
    bulk_copy(smem_u32(sm.recs + buf * kNC), src, bytes, bar);
  }
}

// acc[i][j] += R[K + j] for j < kH.
#define DD_U8_CASE(K)                                                     \
  case K:                                                                 \
    _Pragma("unroll") for (int j = 0; j < kH; ++j) acc[i][j] += R[K + j]; \
    break;

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) fwd_u8_kernel(const U8Params p) {
  extern __shared__ __align__(128) unsigned char smem[];
  Smem sm;
  sm.bar_base = smem_u32(smem);
  sm.recs = reinterpret_cast<Rec*>(smem + 128);
  sm.raw = smem + kRawOffset;
  sm.pw = reinterpret_cast<uint32_t*>(sm.raw + 2 * kNC * static_cast<size_t>(p.lraw));

  const int tid = threadIdx.x;
  const int w = tid >> 5, l = tid & 31;
  const int blk = blockIdx.x % p.n_blocks;
  const int64_t tile = blockIdx.x / p.n_blocks;
  const int64_t t0 = tile * kTile;
  const int n_st = (p.n_chan + kNC - 1) / kNC;

  if (tid == 0) {
    mbar_init(sm.bar_base, kNC + 1);
    mbar_init(sm.bar_base + 8, kNC + 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Base shift of the channel each issuing thread copies, one stage ahead.
  const Rec* my_recs = p.recs + static_cast<int64_t>(blk) * p.n_chan;
  auto base_of = [&](int st) -> int32_t {
    const int c = st * kNC + tid;
    return (tid < kNC && st < n_st && c < p.n_chan) ? my_recs[c].base : 0;
  };
  if (tid <= kNC) {
    issue_stage(p, sm, 0, 0, t0, base_of(0), tid);
    if (n_st > 1) issue_stage(p, sm, 1, 1, t0, base_of(1), tid);
  }
  int32_t next_base = base_of(2);

  uint32_t acc[kDR][kH];
#pragma unroll
  for (int i = 0; i < kDR; ++i)
#pragma unroll
    for (int j = 0; j < kH; ++j) acc[i][j] = 0u;

  bool first_flush = true;
  int chan_done = 0;
  const int units = p.lp >> 2;  // 4 paired words per conversion unit

  for (int st = 0; st < n_st; ++st) {
    const int buf = st & 1;
    const uint32_t parity = (st >> 1) & 1;
    const bool ok = mbar_wait(sm.bar_base + 8u * buf, parity);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(p.err, kErrTimeout);
      // Let any copy still in flight land before the CTA exits (bounded).
      if (tid == 0) {
        mbar_wait(sm.bar_base + 8u * buf, parity);
        if (st + 1 < n_st) mbar_wait(sm.bar_base + 8u * (buf ^ 1), ((st + 1) >> 1) & 1);
      }
      return;
    }
    const int nc = min(kNC, p.n_chan - st * kNC);

    // Re-pack raw bytes into paired 16-bit words: P[k] = X[k] | X[k + 640] << 16.
    {
      const uint8_t* rawb = sm.raw + static_cast<size_t>(buf) * kNC * p.lraw;
      const int total = nc * units;
      for (int u = tid; u < total; u += kThreads) {
        const int ch = static_cast<int>((static_cast<uint64_t>(u) * p.units_magic) >> (32 + p.units_shift));
        const int q = u - ch * units;
        const uint8_t* rc = rawb + static_cast<size_t>(ch) * p.lraw + 4 * q;
        const uint32_t a = *reinterpret_cast<const uint32_t*>(rc);
        const uint32_t b = *reinterpret_cast<const uint32_t*>(rc + kPair);
        const uint32_t t01 = prmt(a, b, 0x5140);
        const uint32_t t23 = prmt(a, b, 0x7362);
        uint4 v;
        v.x = prmt(t01, 0u, 0x4140);
        v.y = prmt(t01, 0u, 0x4342);
        v.z = prmt(t23, 0u, 0x4140);
        v.w = prmt(t23, 0u, 0x4342);
        *reinterpret_cast<uint4*>(sm.pw + static_cast<size_t>(ch) * p.lp + 4 * q) = v;
      }
    }
    __syncthreads();

    // Shift-and-sum: every lane adds its window into its 8 DMs.
    const Rec* rs = sm.recs + buf * kNC;
    for (int ch = 0; ch < nc; ++ch) {
      const uint32_t dl = rs[ch].delta[w];
      const int a = 4 * static_cast<int>(rs[ch].aq[w]);
      const uint4* src = reinterpret_cast<const uint4*>(sm.pw + static_cast<size_t>(ch) * p.lp +
                                                         kH * l + a);
      uint32_t R[kWin];
#pragma unroll
      for (int k = 0; k < kWin / 4; ++k) {
        const uint4 v = src[k];
        R[4 * k] = v.x;
        R[4 * k + 1] = v.y;
        R[4 * k + 2] = v.z;
        R[4 * k + 3] = v.w;
      }
#pragma unroll
      for (int i = 0; i < kDR; ++i) {
        const uint32_t off = (dl >> (4 * i)) & 15u;
        switch (off) {
          DD_U8_CASE(0) DD_U8_CASE(1) DD_U8_CASE(2) DD_U8_CASE(3)
          DD_U8_CASE(4) DD_U8_CASE(5) DD_U8_CASE(6) DD_U8_CASE(7)
          DD_U8_CASE(8) DD_U8_CASE(9) DD_U8_CASE(10) DD_U8_CASE(11)
          DD_U8_CASE(12) DD_U8_CASE(13) DD_U8_CASE(14) DD_U8_CASE(15)
          default: __builtin_unreachable();
        }
      }
    }
    chan_done += nc;
    __syncthreads();  // P, raw[buf] and recs[buf] are free

    if (tid <= kNC && st + 2 < n_st) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_stage(p, sm, st + 2, buf, t0, next_base, tid);
      next_base = base_of(st + 3);
    }

    if ((chan_done & (kFlushChannels - 1)) == 0 || st == n_st - 1) {
      // Widen the 16-bit lanes into the int32 output through a transposed
      // shared-memory tile (index f(p) = p + p / 160 is conflict-free for both
      // the lane-major writes and the row-major reads).
      uint32_t* tr = sm.pw + w * kFlushWords;
      const int wbase = kH * l + (l >> 3);
#pragma unroll
      for (int i = 0; i < kDR; ++i) {
        const int d = blk * kDmCta + w * kDR + i;
#pragma unroll
        for (int j = 0; j < kH; ++j) {
          tr[wbase + j] = acc[i][j] & 0xffffu;
          tr[wbase + j + kPair + 4] = acc[i][j] >> 16;
          acc[i][j] = 0u;
        }
        __syncwarp();
        if (d < p.n_dm) {
          int32_t* row = p.out + static_cast<int64_t>(d) * p.n_out + t0;
          const int64_t lim = p.n_out - t0;
#pragma unroll 8
          for (int k = 0; k < kTile / 32; ++k) {
            const int pos = 32 * k + l;
            if (pos < lim) {
              int32_t v = static_cast<int32_t>(tr[pos + k / 5]);
              if (!first_flush) v += row[pos];
              row[pos] = v;
            }
          }
        }
        __syncwarp();
      }
      first_flush = false;
    }
  }
}

#undef DD_U8_CASE

}  // namespace u8k

int launch_forward_u8(const dd_plan_s* p, const RangePlan& rp, const void* d_in, int64_t stride,
                      int64_t n_samp, int64_t n_out, void* d_out, void* stream) {
  (void)n_samp;
  using namespace u8k;
  U8Params prm{};
  prm.x = static_cast<const uint8_t*>(d_in);
  prm.stride = stride;
  prm.n_chan = p->n_chan;
  prm.recs = reinterpret_cast<const Rec*>(static_cast<const unsigned char*>(p->d_ws) +
                                          rp.off_u8_recs);
  prm.n_dm = static_cast<int32_t>(rp.n_dm);
  prm.n_blocks = rp.u8_n_blocks;
  prm.n_out = n_out;
  prm.lp = rp.u8_lp;
  prm.lraw = rp.u8_lp + kPair;
  prm.units_magic = rp.u8_units_magic;
  prm.units_shift = rp.u8_units_shift;
  prm.out = static_cast<int32_t*>(d_out);
  prm.err = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(p->d_ws) + kStatusOffset);
  const size_t smem = smem_bytes(prm.lp);
  cudaError_t e = cudaFuncSetAttribute(fwd_u8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  const int64_t tiles = (n_out + kTile - 1) / kTile;
  const int64_t grid = tiles * rp.u8_n_blocks;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  fwd_u8_kernel<<<static_cast<unsigned>(grid), kThreads, smem,
                  static_cast<cudaStream_t>(stream)>>>(prm);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace dd
