// fwd_u8.cu -- register-tiled uint8 dedispersion kernel for sm_103a.
//
// Computes Eq. 3 (Algorithm 1) for 8-bit input at time bin 1:
//     Y[d][t] = sum_c X[c][t + s(c, d)]
// exactly (integer sums), with the same output partition as the paper's GPU
// kernel (Sec. 4: a CTA owns D_dm x D_t outputs, threads keep accumulators in
// registers, Algorithm 3) but organised for GB300's issue rate:
//
//  * CTA = W warps x 32 lanes owning dr * W consecutive DMs and 1280 output
//    samples.  Warp w owns DMs d0 + dr*w .. d0 + dr*w + dr - 1; every lane owns
//    the same dr DMs x 40 samples (dr = 8, 6 or 4: the tile shapes of
//    fwd_u8.h, picked per plan).
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
//    channel once (9 x 16-byte shared loads) and adds it into all dr DMs.  The
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
#include "fwd_u8_dispatch.inc"

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
  Rec* recs;           // [2][NC]
  uint8_t* raw;        // [2][NC][lraw]
  uint32_t* pw;        // [NC][lp]
};

// Issue the TMA copies of stage `st` into buffer `buf`.  Threads 0..NC-1 copy
// one channel each, thread NC copies the stage's records.
template <int kNC>
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

static_assert(kH == 20 && kWin == 36 && kMaxOff == 15,
              "fwd_u8_dispatch.inc is generated for 20 words, a 36-word window and 16 offsets");

}  // namespace

// Adds the lane's window slices into its DR register tiles: one warp-uniform
// indexed branch per DM (fwd_u8_dispatch.inc, generated by gen_u8_dispatch.py).
template <int DR>
__device__ __forceinline__ void dispatch_dms(uint32_t (&acc)[DR][kH], const uint32_t (&R)[kWin],
                                             uint32_t dl) {
  uint32_t ix[DR];
#pragma unroll
  for (int i = 0; i < DR; ++i) ix[i] = (dl >> (4 * i)) & 15u;
  if constexpr (DR == 4) {
    DD_U8_CHANNEL_4(acc, R, ix);
  } else if constexpr (DR == 6) {
    DD_U8_CHANNEL_6(acc, R, ix);
  } else {
    static_assert(DR == 8, "tile shapes are 4, 6 or 8 DMs per lane");
    DD_U8_CHANNEL_8(acc, R, ix);
  }
}

template <int DR, int NW, int MINB, int kNC>
__global__ void __launch_bounds__(NW * 32, MINB) fwd_u8_kernel(const U8Params p) {
  constexpr int kThreads = NW * 32;
  constexpr int kDmCta = DR * NW;
  constexpr int kDR = DR;
  static_assert(NW * kFlushWords <= kNC * 672, "flush tile must fit the paired window buffer");
  extern __shared__ __align__(128) unsigned char smem[];
  Smem sm;
  sm.bar_base = smem_u32(smem);
  sm.recs = reinterpret_cast<Rec*>(smem + kRecOffset);
  constexpr size_t kRawOff = raw_offset(kNC);
  sm.raw = smem + kRawOff;
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
    issue_stage<kNC>(p, sm, 0, 0, t0, base_of(0), tid);
    if (n_st > 1) issue_stage<kNC>(p, sm, 1, 1, t0, base_of(1), tid);
  }
  int32_t next_base = base_of(2);

  uint32_t acc[kDR][kH];
#pragma unroll
  for (int i = 0; i < kDR; ++i)
#pragma unroll
    for (int j = 0; j < kH; ++j) acc[i][j] = 0u;

  bool first_flush = true;
  int since_flush = 0;  // channels added into the 16-bit lanes since the last widen
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

    // Shift-and-sum: every lane adds its window into its DR DMs.  One indexed
    // branch per DM selects the register slice R[off .. off + 20) (see
    // gen_u8_dispatch.py); the loop is kept rolled so the dispatch block, and
    // its PTX labels, appears once per kernel.
    const Rec* rs = sm.recs + buf * kNC;
#pragma unroll 1
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
      dispatch_dms<DR>(acc, R, dl);
    }
    since_flush += nc;
    __syncthreads();  // P, raw[buf] and recs[buf] are free

    if (tid <= kNC && st + 2 < n_st) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_stage<kNC>(p, sm, st + 2, buf, t0, next_base, tid);
      next_base = base_of(st + 3);
    }

    // Widen before the next stage could take a lane past kFlushChannels channels.
    if (since_flush + kNC > kFlushChannels || st == n_st - 1) {
      since_flush = 0;
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
          // Two halves of 20 positions: issue all loads of a half before any add.
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            int32_t v[kTile / 64];
#pragma unroll
            for (int k = 0; k < kTile / 64; ++k) {
              const int kk = h * (kTile / 64) + k;
              v[k] = static_cast<int32_t>(tr[32 * kk + l + kk / 5]);
            }
            if (!first_flush) {
              int32_t g[kTile / 64];
#pragma unroll
              for (int k = 0; k < kTile / 64; ++k) {
                const int pos = 32 * (h * (kTile / 64) + k) + l;
                g[k] = pos < lim ? __ldcg(row + pos) : 0;
              }
#pragma unroll
              for (int k = 0; k < kTile / 64; ++k) v[k] += g[k];
            }
#pragma unroll
            for (int k = 0; k < kTile / 64; ++k) {
              const int pos = 32 * (h * (kTile / 64) + k) + l;
              if (pos < lim) row[pos] = v[k];
            }
          }
        }
        __syncwarp();
      }
      first_flush = false;
    }
  }
}


}  // namespace u8k

namespace {

template <int DR, int NW, int MINB, int NC>
int launch_shape(const u8k::U8Params& prm, int64_t grid, cudaStream_t st) {
  const u8k::Shape* sh = u8k::shape_for(DR);
  const size_t smem = u8k::smem_bytes(*sh, prm.lp);
  auto kern = u8k::fwd_u8_kernel<DR, NW, MINB, NC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  kern<<<static_cast<unsigned>(grid), NW * 32, smem, st>>>(prm);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace

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
  const int64_t tiles = (n_out + kTile - 1) / kTile;
  const int64_t grid = tiles * rp.u8_n_blocks;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (rp.u8_dr) {
    case 8: return launch_shape<8, 8, 1, 16>(prm, grid, st);
    case 6: return launch_shape<6, 12, 1, 24>(prm, grid, st);
    case 4: return launch_shape<4, 8, 2, 16>(prm, grid, st);
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

int launch_forward_u8_with_tables(const dd_plan_s* p, const RangePlan& rp, const void* recs,
                                  int32_t* err, const void* d_in, int64_t stride,
                                  int64_t n_out, void* d_out, void* stream) {
  using namespace u8k;
  U8Params prm{};
  prm.x = static_cast<const uint8_t*>(d_in);
  prm.stride = stride;
  prm.n_chan = p->n_chan;
  prm.recs = static_cast<const Rec*>(recs);
  prm.n_dm = static_cast<int32_t>(rp.n_dm);
  prm.n_blocks = rp.u8_n_blocks;
  prm.n_out = n_out;
  prm.lp = rp.u8_lp;
  prm.lraw = rp.u8_lp + kPair;
  prm.units_magic = rp.u8_units_magic;
  prm.units_shift = rp.u8_units_shift;
  prm.out = static_cast<int32_t*>(d_out);
  prm.err = err;
  const int64_t tiles = (n_out + kTile - 1) / kTile;
  const int64_t grid = tiles * rp.u8_n_blocks;
  if (grid <= 0 || grid > 0x7fffffffLL) return static_cast<int>(cudaErrorInvalidConfiguration);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (rp.u8_dr) {
    case 8: return launch_shape<8, 8, 1, 16>(prm, grid, st);
    case 6: return launch_shape<6, 12, 1, 24>(prm, grid, st);
    case 4: return launch_shape<4, 8, 2, 16>(prm, grid, st);
  }
  return static_cast<int>(cudaErrorInvalidValue);
}

}  // namespace dd
