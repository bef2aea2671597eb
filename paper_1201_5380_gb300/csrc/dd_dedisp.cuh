// Direct dedispersion kernel (Sec. 2, Eq. 2) for sm_103a.
//
// One thread block owns a tile of B = NWARP*DPW adjacent trials x T output
// samples of one work item and walks the channels in chunks of `cc`, a size
// the host picks per trial block (as many channels as the block's windows
// leave room for in shared memory).  For
// each chunk it stages, per channel, the window of the channel's image row
// that any of its B trials needs (the temporal caching of Sec. 2.3, the
// staged tile serving the whole trial block), as SPW copies shifted by one
// lane each, so that for every (trial, channel) pair a warp reads its 32*K
// words with plain conflict-free 32-bit shared loads at a word-aligned
// offset.  Lanes of a word are summed lane-parallel (the bit-level
// parallelism of Sec. 2.3): 4-bit lanes take 4 channels of 2-bit data (5
// fit, 85 in 8-bit lanes), then widen to 8-, 16- and if needed 32-bit lanes,
// so integer sums stay exact.  The kill mask is folded into the image
// (masked rows are zero), the arithmetic form of Sec. 2.3.
//
// Lane layout: warp w handles trials d0 + w*DPW + i (i < DPW); lane l handles
// words l + 32*j (j < K) of the tile, i.e. samples t0 + SPW*(l+32j) + 0..SPW-1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dd_internal.h"

namespace dd {

template <int FMT> struct FmtT;
template <> struct FmtT<FMT_NIB> { static constexpr int SPW = 8, LW = 4; };
template <> struct FmtT<FMT_BYTE> { static constexpr int SPW = 4, LW = 8; };
template <> struct FmtT<FMT_HALF> { static constexpr int SPW = 2, LW = 16; };
template <> struct FmtT<FMT_U32> { static constexpr int SPW = 1, LW = 32; };
template <> struct FmtT<FMT_F32> { static constexpr int SPW = 1, LW = 32; };
template <> struct FmtT<FMT_TRI> { static constexpr int SPW = 3, LW = 10; };
template <> struct FmtT<FMT_SB8> { static constexpr int SPW = 4, LW = 8; };

// Word w of a staged row shifted by kap samples (the next word b supplies
// the samples shifted in): a funnel shift for lanes that fill the word, an
// explicit merge for the 10-bit lanes (bits 30-31 stay zero).
template <int FMT>
__device__ __forceinline__ uint32_t lane_shift(uint32_t a, uint32_t b, int kap) {
  if constexpr (FMT == FMT_TRI) {
    return kap == 1 ? (a >> 10) | ((b << 20) & 0x3FF00000u) : (a >> 20) | ((b << 10) & 0x3FFFFC00u);
  } else {
    return __funnelshift_r(a, b, kap * FmtT<FMT>::LW);
  }
}

// ---------------------------------------------------------------------------
// Per-word accumulators.  flush0/1/2 move a level into the next wider one;
// final() returns the SPW exact sums of the word in time order.
// ---------------------------------------------------------------------------
template <int FMT, bool WIDE> struct Acc;

// 4-bit lanes: n holds samples 0..7 of the word.  b0 = samples {0,2,4,6} and
// b1 = {1,3,5,7} in 8-bit lanes; h0 = {0,4}, h1 = {2,6}, h2 = {1,5},
// h3 = {3,7} in 16-bit lanes; u[] = 32-bit sums when WIDE.
template <bool WIDE> struct Acc<FMT_NIB, WIDE> {
  uint32_t n, b0, b1, h0, h1, h2, h3;
  uint32_t u[WIDE ? 8 : 1];
  __device__ __forceinline__ void zero() {
    n = b0 = b1 = h0 = h1 = h2 = h3 = 0u;
#pragma unroll
    for (int i = 0; i < (WIDE ? 8 : 1); ++i) u[i] = 0u;
  }
  __device__ __forceinline__ void add4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    n = n + x0 + x1;
    n = n + x2 + x3;
  }
  __device__ __forceinline__ void flush0() {
    b0 += n & 0x0F0F0F0Fu;
    b1 += (n >> 4) & 0x0F0F0F0Fu;
    n = 0u;
  }
  // Two groups of four channels whose 4-bit sums each fit a nibble (f0 ==
  // 1), widened to the 8-bit lanes together: one add per lane set for both.
  // The odd nibbles are not masked here: b1 takes the plain sum of a >> 4,
  // which is the odd nibbles in their byte lanes plus the even nibbles of
  // bytes 1..3 four bits up, i.e. b1 + ((b0 & 0xFFFFFF00) >> 4) (mod 2^32);
  // pair_fix() takes the second part back out before a flush.
  __device__ __forceinline__ void add8_flush(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                             uint32_t x4, uint32_t x5, uint32_t x6,
                                             uint32_t x7) {
    const uint32_t a = (x0 + x1) + (x2 + x3);
    const uint32_t c = (x4 + x5) + (x6 + x7);
    b0 += (a & 0x0F0F0F0Fu) + (c & 0x0F0F0F0Fu);
    b1 += (a >> 4) + (c >> 4);
  }
  __device__ __forceinline__ void pair_fix() { b1 -= (b0 & 0xFFFFFF00u) >> 4; }
  __device__ __forceinline__ void flush1() {
    h0 += b0 & 0x00FF00FFu;
    h1 += (b0 >> 8) & 0x00FF00FFu;
    h2 += b1 & 0x00FF00FFu;
    h3 += (b1 >> 8) & 0x00FF00FFu;
    b0 = b1 = 0u;
  }
  __device__ __forceinline__ void flush2() {
    if (WIDE) {
      u[0] += h0 & 0xFFFFu; u[4] += h0 >> 16;
      u[2] += h1 & 0xFFFFu; u[6] += h1 >> 16;
      u[1] += h2 & 0xFFFFu; u[5] += h2 >> 16;
      u[3] += h3 & 0xFFFFu; u[7] += h3 >> 16;
      h0 = h1 = h2 = h3 = 0u;
    }
  }
  __device__ __forceinline__ void final(uint32_t v[8]) {
    flush0();
    flush1();
    if (WIDE) {
      flush2();
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = u[WIDE ? i : 0];
    } else {
      v[0] = h0 & 0xFFFFu; v[4] = h0 >> 16;
      v[2] = h1 & 0xFFFFu; v[6] = h1 >> 16;
      v[1] = h2 & 0xFFFFu; v[5] = h2 >> 16;
      v[3] = h3 & 0xFFFFu; v[7] = h3 >> 16;
    }
  }
};

// 8-bit lanes: b holds samples 0..3; h0 = {0,2}, h1 = {1,3} in 16-bit lanes.
template <bool WIDE> struct Acc<FMT_BYTE, WIDE> {
  uint32_t b, h0, h1;
  uint32_t u[WIDE ? 4 : 1];
  __device__ __forceinline__ void zero() {
    b = h0 = h1 = 0u;
#pragma unroll
    for (int i = 0; i < (WIDE ? 4 : 1); ++i) u[i] = 0u;
  }
  __device__ __forceinline__ void add4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    b = b + x0 + x1;
    b = b + x2 + x3;
  }
  __device__ __forceinline__ void flush0() {
    h0 += b & 0x00FF00FFu;
    h1 += (b >> 8) & 0x00FF00FFu;
    b = 0u;
  }
  __device__ __forceinline__ void flush1() {
    if (WIDE) {
      u[0] += h0 & 0xFFFFu; u[2] += h0 >> 16;
      u[1] += h1 & 0xFFFFu; u[3] += h1 >> 16;
      h0 = h1 = 0u;
    }
  }
  __device__ __forceinline__ void flush2() {}
  __device__ __forceinline__ void final(uint32_t v[4]) {
    flush0();
    if (WIDE) {
      flush1();
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = u[WIDE ? i : 0];
    } else {
      v[0] = h0 & 0xFFFFu; v[2] = h0 >> 16;
      v[1] = h1 & 0xFFFFu; v[3] = h1 >> 16;
    }
  }
};

// 16-bit lanes: h holds samples 0..1.
template <bool WIDE> struct Acc<FMT_HALF, WIDE> {
  uint32_t h;
  uint32_t u[WIDE ? 2 : 1];
  __device__ __forceinline__ void zero() {
    h = 0u;
#pragma unroll
    for (int i = 0; i < (WIDE ? 2 : 1); ++i) u[i] = 0u;
  }
  __device__ __forceinline__ void add4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    h = h + x0 + x1;
    h = h + x2 + x3;
  }
  __device__ __forceinline__ void flush0() {
    if (WIDE) {
      u[0] += h & 0xFFFFu;
      u[WIDE ? 1 : 0] += h >> 16;
      h = 0u;
    }
  }
  __device__ __forceinline__ void flush1() {}
  __device__ __forceinline__ void flush2() {}
  __device__ __forceinline__ void final(uint32_t v[2]) {
    if (WIDE) {
      flush0();
      v[0] = u[0];
      v[1] = u[WIDE ? 1 : 0];
    } else {
      v[0] = h & 0xFFFFu;
      v[1] = h >> 16;
    }
  }
};

// 8-bit lanes of sub-band stage 2 (FMT_SB8): every staged value is a
// stage-1 sum below 128, so two sub-bands add lane-parallel without a carry
// (a pair stays below 256).  Each pair is then spread into 16-bit lanes:
// e = samples {0,2} (a mask), o = samples {1,3} (a byte permute).  Exact
// while a trial's total stays below 2^16, which the plan checks; there is
// no wide variant.
template <bool WIDE> struct Acc<FMT_SB8, WIDE> {
  uint32_t e, o;
  __device__ __forceinline__ void zero() { e = o = 0u; }
  __device__ __forceinline__ void add4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    const uint32_t a = x0 + x1, c = x2 + x3;
    e = e + (a & 0x00FF00FFu) + (c & 0x00FF00FFu);
    // bytes 1 and 3 of the pair into the low bytes of the 16-bit lanes
    o = o + __byte_perm(a, 0u, 0x4341u) + __byte_perm(c, 0u, 0x4341u);
  }
  __device__ __forceinline__ void flush0() {}
  __device__ __forceinline__ void flush1() {}
  __device__ __forceinline__ void flush2() {}
  __device__ __forceinline__ void final(uint32_t v[4]) {
    v[0] = e & 0xFFFFu; v[2] = e >> 16;
    v[1] = o & 0xFFFFu; v[3] = o >> 16;
  }
};

template <bool WIDE> struct Acc<FMT_U32, WIDE> {
  uint32_t s;
  __device__ __forceinline__ void zero() { s = 0u; }
  __device__ __forceinline__ void add4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    s = s + x0 + x1;
    s = s + x2 + x3;
  }
  __device__ __forceinline__ void flush0() {}
  __device__ __forceinline__ void flush1() {}
  __device__ __forceinline__ void flush2() {}
  __device__ __forceinline__ void final(uint32_t v[1]) { v[0] = s; }
};

// 10-bit lanes: a word holds samples 0..2 in bits [0,10), [10,20),
// [20,30).  Four channels of 8-bit samples fit a lane (4 * 255 < 1024), so
// a group of four is summed lane-parallel into a.  Then:
//   z += a                the plain 32-bit sum of every group: lanes carry
//                         into each other, modulo 2^32
//   w += a & 0x3FF003FF   lanes 0 and 2 apart: lane 0 in [0,20) for the
//                         whole item (nchans * 255 < 2^20), lane 2 in
//                         [20,32) for four groups, then moved into u2
// and lane 1 is what z holds beyond lanes 0 and 2:
// (z - lane0 - lane2 * 2^20) mod 2^32 = lane1 * 2^10, exact since
// lane1 < 2^22.  The plan stages 10-bit lanes for at most 4112 channels.
template <bool WIDE> struct Acc<FMT_TRI, WIDE> {
  uint32_t z, w, u2;
  __device__ __forceinline__ void zero() { z = w = u2 = 0u; }
  __device__ __forceinline__ void add4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    const uint32_t a = (x0 + x1) + (x2 + x3);
    z += a;
    w += a & 0x3FF003FFu;
  }
  __device__ __forceinline__ void flush0() {}
  // two groups of four channels (lane 2 of w then holds two such pairs)
  __device__ __forceinline__ void add8(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                       uint32_t x4, uint32_t x5, uint32_t x6, uint32_t x7) {
    const uint32_t a = (x0 + x1) + (x2 + x3);
    const uint32_t c = (x4 + x5) + (x6 + x7);
    z = z + a + c;
    w = w + (a & 0x3FF003FFu) + (c & 0x3FF003FFu);
  }
  // every four groups
  __device__ __forceinline__ void flush1() {
    u2 += w >> 20;
    w &= 0xFFFFFu;
  }
  __device__ __forceinline__ void flush2() {}
  __device__ __forceinline__ void final(uint32_t v[3]) {
    flush1();
    v[0] = w;
    v[1] = (z - w - (u2 << 20)) >> 10;
    v[2] = u2;
  }
};

// Float: channels are summed into a partial over 32 channels (8 groups),
// then the partial is added into the total (bounds the FP32 error to about
// 64 ulp of sum|A| rather than 1024).
template <bool WIDE> struct Acc<FMT_F32, WIDE> {
  float p, s;
  __device__ __forceinline__ void zero() { p = s = 0.f; }
  __device__ __forceinline__ void add4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    p = __fadd_rn(p, __uint_as_float(x0));
    p = __fadd_rn(p, __uint_as_float(x1));
    p = __fadd_rn(p, __uint_as_float(x2));
    p = __fadd_rn(p, __uint_as_float(x3));
  }
  __device__ __forceinline__ void flush0() {
    s = __fadd_rn(s, p);
    p = 0.f;
  }
  __device__ __forceinline__ void flush1() {}
  __device__ __forceinline__ void flush2() {}
  __device__ __forceinline__ void final(uint32_t v[1]) {
    flush0();
    v[0] = __float_as_uint(s);
  }
};

__device__ __forceinline__ int find_seg(const LaunchParams& p, int64_t item) {
  int lo = 0, hi = p.n_segs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (p.segs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// TMA (bulk async copy) and mbarrier helpers.  Every wait is bounded: after
// kWaitLimit polls the kernel records DEV_TIMEOUT and carries on, so a lost
// transfer can never hang the GPU.
// ---------------------------------------------------------------------------
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void* src, uint32_t bytes,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// Window start (image word, multiple of 4) of a channel whose first trial
// has delay s0, for a tile starting at output time t0.
template <int SPW>
__device__ __forceinline__ int64_t window_word(int64_t t0, int32_t s0, int lo_slack) {
  const int64_t b = t0 + kPad + (int64_t)s0 - lo_slack;  // >= 0 (kPad >= lo_slack)
  return (b / (4 * SPW)) * 4;
}

// Shared-memory layout (32-bit words):
//   [0,4)            two mbarriers
//   two buffers, each
//     landing[cc][nww+4]           TMA destination: raw image windows, read
//                                  by the sums as the unshifted copy
//     copies [cc*(SPW-1)][nww]     the other SPW-1 lane-shifted copies of
//                                  each window
//   addr   [2][B*cc]               byte offset of each (trial, channel)
//                                  window inside its buffer (lane 0, word 0)
//
// The staging tables are built on the host per plan and geometry (they do
// not depend on the time tile): per trial block its chunk size cc and window
// width nww (the layout above, so each block stages as many channels per
// chunk as its own windows allow), per (trial block, channel) the window
// start and the words its trials read, and per (trial block, chunk) the
// B x cc window offsets, which arrive by TMA with the chunk's windows.
//
// Per chunk (cc channels) of an item, one __syncthreads:
//   prefetch the next chunk's window records -> registers
//   wait for this chunk's TMA; build its shifted copies (as far as read)
//   __syncthreads
//   warp 0 issues the next chunk's TMA (windows + offsets)
//   shift-and-sum this chunk
// PBG: each trial block has its own chunk geometry (read from its staging
// tables); otherwise the launch's (every block of the launch has the same).
// k_dedisp stages one time tile per work item; k_dedisp_mt is the same body
// for items of several consecutive tiles of one trial block (the sub-band
// stages' one- or two-chunk items), see dd_dedisp_body.cuh.

#define DD_KERNEL k_dedisp
#define DD_MT 0
#include "dd_dedisp_body.cuh"
#undef DD_KERNEL
#undef DD_MT

#define DD_KERNEL k_dedisp_mt
#define DD_MT 1
#include "dd_dedisp_body.cuh"
#undef DD_KERNEL
#undef DD_MT

// Host helpers used by the per-format translation units.
template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG, bool MT>
auto kernel_of() {
  if constexpr (MT)
    return k_dedisp_mt<FMT, OUTK, WIDE, NWARP, DPW, K, PBG>;
  else
    return k_dedisp<FMT, OUTK, WIDE, NWARP, DPW, K, PBG>;
}

template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG, bool MT>
cudaError_t launch_one(const LaunchParams& p, int grid, size_t smem, cudaStream_t st) {
  auto kern = kernel_of<FMT, OUTK, WIDE, NWARP, DPW, K, PBG, MT>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NWARP * 32, smem, st>>>(p);
  return cudaGetLastError();
}

template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG, bool MT>
cudaError_t occupancy_one(size_t smem, int* nblk) {
  auto kern = kernel_of<FMT, OUTK, WIDE, NWARP, DPW, K, PBG, MT>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nblk, kern, NWARP * 32, smem);
}

template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG, bool MT = false>
cudaError_t run_one(const LaunchParams* p, int grid, size_t smem, cudaStream_t st, int* occ) {
  return occ ? occupancy_one<FMT, OUTK, WIDE, NWARP, DPW, K, PBG, MT>(smem, occ)
             : launch_one<FMT, OUTK, WIDE, NWARP, DPW, K, PBG, MT>(*p, grid, smem, st);
}

// The multi-tile kernel of one (FMT, OUTK, WIDE) and tile shape I (compiled
// only for the shapes the sub-band stages run, see multi_tile_compiled).
template <int FMT, int OUTK, bool WIDE, int I>
cudaError_t dispatch_mt(bool pbg, const LaunchParams* p, int grid, size_t smem, cudaStream_t st,
                        int* occ) {
  constexpr int NW = kTileCfgs[I].nwarp, DP = kTileCfgs[I].dpw, KK = kTileCfgs[I].k;
  return pbg ? run_one<FMT, OUTK, WIDE, NW, DP, KK, true, true>(p, grid, smem, st, occ)
             : run_one<FMT, OUTK, WIDE, NW, DP, KK, false, true>(p, grid, smem, st, occ);
}

// Dispatch over the compiled tile shapes (and the per-block geometry
// variant) for one (FMT, OUTK, WIDE).
template <int FMT, int OUTK, bool WIDE>
cudaError_t dispatch_cfg(int cfg, bool pbg, const LaunchParams* p, int grid, size_t smem,
                         cudaStream_t st, int* occ) {
  switch (cfg) {
#define DD_CFG_CASE(I)                                                                   \
  case I:                                                                                \
    return pbg ? run_one<FMT, OUTK, WIDE, kTileCfgs[I].nwarp, kTileCfgs[I].dpw,          \
                         kTileCfgs[I].k, true>(p, grid, smem, st, occ)                   \
               : run_one<FMT, OUTK, WIDE, kTileCfgs[I].nwarp, kTileCfgs[I].dpw,          \
                         kTileCfgs[I].k, false>(p, grid, smem, st, occ);
    DD_CFG_CASE(0)
    DD_CFG_CASE(1)
    DD_CFG_CASE(2)
    DD_CFG_CASE(3)
    DD_CFG_CASE(4)
    case 5:
      // 16 words a lane: only where a word's accumulators take one or two
      // registers (the other formats would spill)
      if constexpr (FmtT<FMT>::SPW <= 2) {
        return pbg ? run_one<FMT, OUTK, WIDE, 16, 2, 16, true>(p, grid, smem, st, occ)
                   : run_one<FMT, OUTK, WIDE, 16, 2, 16, false>(p, grid, smem, st, occ);
      } else {
        return cudaErrorInvalidValue;
      }
#undef DD_CFG_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace dd
