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
template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG>
__global__ void __launch_bounds__(NWARP * 32, (NWARP <= 8 ? 2 : 1)) k_dedisp(const LaunchParams p) {
  constexpr int SPW = FmtT<FMT>::SPW;
  constexpr int LW = FmtT<FMT>::LW;
  constexpr int NT = NWARP * 32;
  constexpr int B = NWARP * DPW;
  constexpr int T = 32 * K * SPW;

  extern __shared__ uint4 smem4[];
  uint32_t* const sm = reinterpret_cast<uint32_t*>(smem4);
  const uint32_t sm_base = smem_addr(sm);
  const uint32_t bar0 = sm_base;    // two 8-byte mbarriers at word 0 and 2
  // one sample per word needs no shifted copies: lanes read the landing area
  constexpr bool COPIES = SPW > 1;
  uint32_t* const landing = sm + 4;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;

  // Chunk geometry and the staging layout it implies: the launch's, set up
  // once here, or (PBG) each trial block's, set up per work item.
  struct Geo {
    int cc, cc_log, nww, nwl, buf_words, n_entries, tpc_log, bc;
    uint32_t* s_addr;
  };
  auto make_geo = [&](int cc, int nww) {
    Geo g;
    g.cc = cc;  // power of two, 4..32
    g.cc_log = 31 - __clz(cc);
    g.nww = nww;  // window words (multiple of 4)
    g.nwl = nww + 4;
    // one buffer: the landing windows (the sums read them as the unshifted
    // copy), then the SPW-1 shifted copies built from them
    g.buf_words = cc * g.nwl + (COPIES ? cc * (SPW - 1) * nww : 0);
    g.s_addr = landing + 2 * g.buf_words;
    g.n_entries = B << g.cc_log;  // offsets per chunk
    // the builder threads of a channel: NT / cc of them
    g.tpc_log = (31 - __clz(NT)) - g.cc_log;
    g.bc = tid >> g.tpc_log;
    return g;
  };
  const Geo geo_launch = make_geo(PBG ? 4 : p.cc, PBG ? 0 : p.nww);

  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();

  uint32_t kk = 0;  // chunks consumed by this block (buffer = kk & 1, parity = (kk >> 1) & 1)

  // next work item: from the launch's counter (neighbouring items run
  // together), else the static grid stride
  __shared__ long long s_next_item;
  auto next_item = [&](int64_t cur) -> int64_t {
    if (!p.next_item) return cur + gridDim.x;
    __syncthreads();  // every thread has read the previous value
    if (tid == 0)
      s_next_item = (long long)gridDim.x + (long long)atomicAdd(p.next_item, 1ull);
    __syncthreads();
    return s_next_item;
  };

  for (int64_t item = blockIdx.x; item < p.n_items; item = next_item(item)) {
    const Seg& S = p.segs[find_seg(p, item)];
    const int64_t li = item - S.item_begin;
    const int n_dmblk = S.n_dmblk;
    const int64_t per_tile = (int64_t)S.n_groups * n_dmblk;
    const int64_t lt = li / per_tile;
    const int64_t tile = S.tile0 + lt;
    const int64_t rem = li - lt * per_tile;
    const int grp = (int)(rem / n_dmblk);
    const int blk = (int)(rem - (int64_t)grp * n_dmblk);
    const int ndm_g = (grp == S.n_groups - 1) ? S.ndm_last : S.ndm;
    // this item's staging tables: the trial block's chunk geometry, then one
    // window record per channel (a per-block geometry load is issued here,
    // beside the block-start loads, rather than after them)
    const int nchan = S.nchan;
    const int2* __restrict__ crec_g =
        reinterpret_cast<const int2*>(S.crec + (int64_t)grp * S.g_crec);
    const int2* __restrict__ crec = crec_g + (int64_t)blk * nchan;
    int2 bgeo = make_int2(0, 0);
    if constexpr (PBG) bgeo = __ldg(&crec_g[(int64_t)n_dmblk * nchan + blk]);
    int d0, nd;
    if (S.blk) {
      const int32_t* bt = S.blk + (int64_t)grp * (n_dmblk + 1);
      d0 = __ldg(&bt[blk]);
      nd = min(B, __ldg(&bt[blk + 1]) - d0);
      if (nd == 0) continue;  // padding block of a group with fewer blocks
    } else {
      d0 = blk * B;
      nd = min(B, ndm_g - d0);
    }
    const int64_t t0 = tile * T;
    const int64_t t_end = min(t0 + T, S.nsamps);
    const int64_t row_words = S.row_words;
    const uint32_t* __restrict__ img = S.img + (int64_t)grp * S.g_img;
    uint32_t* const out_g = reinterpret_cast<uint32_t*>(S.out) + (int64_t)grp * S.g_out;
    if (nd <= 0 || t0 >= S.nsamps) {
      if (tid == 0) atomicOr(p.status, DEV_BAD_ITEM);
      continue;
    }
    const Geo G = PBG ? make_geo(bgeo.x, bgeo.y) : geo_launch;
    const int cc = G.cc, cc_log = G.cc_log, nww = G.nww, nwl = G.nwl;
    uint32_t* const s_addr = G.s_addr;
    const int buf_words = G.buf_words;
    const int n_entries = G.n_entries, tpc_log = G.tpc_log, bc = G.bc;
    const int nchunks = (nchan + cc - 1) >> cc_log;
    const uint32_t* __restrict__ atab =
        S.atab + (int64_t)grp * S.g_atab + (int64_t)blk * S.atab_blk;
    const int64_t t0w = t0 / SPW;  // image word of time t0 - kPad

    // window record of channel c0 + (warp 0: lane; builders: bc) of chunk k
    auto rec_of = [&](int k, int c) -> int2 {
      const int ca = (k << cc_log) + c;
      return ca < nchan ? __ldg(&crec[ca]) : make_int2(0, 32 * K);
    };
    // TMA of chunk k (warp 0): the offsets, then each channel's window.  A
    // window running past the end of its row (a launch over images of
    // different lengths) is shortened: those words are beyond every valid
    // output of this image.
    auto issue = [&](int k, int nb, int2 r) {
      const uint32_t bar = bar0 + 8u * nb;
      const int c0 = k << cc_log;
      const int cabs = min(c0 + lane, nchan - 1);
      int64_t wi = t0w + r.x;
      const bool has = lane < cc && c0 + lane < nchan;
      if (has && (wi < 0 || wi + 4 > row_words)) {
        atomicOr(p.status, DEV_BAD_READ);
        wi = 0;
      }
      // the words this channel's trials read (plus the next word, which the
      // lane-shift build reads), not the block's whole window
      const int64_t want = min((int64_t)nwl, (int64_t)((r.y + 4 + 3) & ~3));
      const uint32_t words = has ? (uint32_t)min(want, row_words - wi) : 0u;
      const uint32_t tab_bytes = (uint32_t)n_entries * 4u;
      const uint32_t total = __reduce_add_sync(0xffffffffu, words * 4u) + tab_bytes;
      // No proxy fence here: the copies overwrite words that the block only
      // read since they last landed (ordered by the barrier), except the
      // zero-filled windows of channels past the band, whose writers fence
      // before that barrier.
      if (lane == 0) {
        mbar_arrive_expect_tx(bar, total);
        tma_load_1d(smem_addr(s_addr + nb * n_entries), atab + (int64_t)k * n_entries, tab_bytes,
                    bar);
      }
      __syncwarp();
      if (words) {
        tma_load_1d(smem_addr(landing + nb * buf_words + lane * nwl),
                    img + (int64_t)cabs * row_words + wi, words * 4u, bar);
      }
    };

    // pairs of 4-channel groups per step (the item's chunk size allows it)
    bool paired = false;
    if constexpr (FMT == FMT_NIB)
      paired = p.f0 == 1 && p.f1 >= 2 && (cc & 7) == 0 && (cc >> 3) <= (p.f1 >> 1);
    if constexpr (FMT == FMT_TRI) paired = (cc & 7) == 0;

    Acc<FMT, WIDE> acc[DPW][K];
#pragma unroll
    for (int i = 0; i < DPW; ++i)
#pragma unroll
      for (int j = 0; j < K; ++j) acc[i][j].zero();
    int g0 = 0, g1 = 0, g2 = 0;

    // prologue: chunk 0
    int2 rec_w = make_int2(0, 0);  // warp 0: window record of the next chunk to issue
    if (warp == 0) issue(0, kk & 1, rec_of(0, lane));
    int span = COPIES ? rec_of(0, bc).y : 0;  // builders: words of this chunk's window

    for (int k = 0; k < nchunks; ++k, ++kk) {
      const int buf = kk & 1;
      const int c0 = k << cc_log;
      const bool more = k + 1 < nchunks;
      int span_next = 0;
      if (more) {
        if (warp == 0) rec_w = rec_of(k + 1, lane);
        if (COPIES) span_next = rec_of(k + 1, bc).y;
      }
      // (a) wait for the chunk's windows and offsets, then build the SPW
      //     shifted copies as far as the chunk's trials read
      if (!mbar_wait_bounded(bar0 + 8u * buf, (kk >> 1) & 1u)) {
        atomicOr(p.status, DEV_TIMEOUT);
        mbar_wait_bounded(bar0 + 8u * buf, (kk >> 1) & 1u);
      }
      if (!COPIES) {
        if (c0 + cc > nchan) {
          uint32_t* const land = landing + buf * buf_words;
          for (int e = tid; e < (c0 + cc - nchan) * nwl; e += NT)
            land[(nchan - c0) * nwl + e] = 0u;
          // a later bulk copy (async proxy) may land on these words
          fence_proxy_async_smem();
        }
      } else {
        uint32_t* const land = landing + buf * buf_words;
        uint32_t* const cp = land + cc * nwl;
        const int c = bc;
        const int nq = (min(span, nww) + 3) >> 2;
        const bool live = c0 + c < nchan;
        for (int q = tid & ((1 << tpc_log) - 1); q < nq; q += (1 << tpc_log)) {
          uint4 w = make_uint4(0u, 0u, 0u, 0u);
          uint32_t w4 = 0u;
          if (live) {
            w = *reinterpret_cast<const uint4*>(land + c * nwl + 4 * q);
            w4 = land[c * nwl + 4 * q + 4];
          } else {
            // a channel past the band: its (never copied) window reads zero
            *reinterpret_cast<uint4*>(land + c * nwl + 4 * q) = w;
          }
          uint32_t* dst = cp + c * (SPW - 1) * nww + 4 * q;
#pragma unroll
          for (int kap = 1; kap < SPW; ++kap) {
            uint4 v;
            v.x = lane_shift<FMT>(w.x, w.y, kap);
            v.y = lane_shift<FMT>(w.y, w.z, kap);
            v.z = lane_shift<FMT>(w.z, w.w, kap);
            v.w = lane_shift<FMT>(w.w, w4, kap);
            *reinterpret_cast<uint4*>(dst + (kap - 1) * nww) = v;
          }
        }
        // a later bulk copy (async proxy) may land on the zeroed words
        if (!live) fence_proxy_async_smem();
      }
      __syncthreads();
      // (b) next chunk's TMA (its buffers were released by the barrier above)
      if (more && warp == 0) issue(k + 1, buf ^ 1, rec_w);
      span = span_next;
      // (c) shift-and-sum over the chunk, four channels per group
      const uint32_t* const sa = s_addr + buf * n_entries;
      const uint32_t lane_off = smem_addr(landing + buf * buf_words) + (uint32_t)lane * 4u;
      if (warp * DPW >= nd) {
        // every trial slot of this warp is past the block's last trial: its
        // sums would be discarded (a short last block, a short sub-band
        // group), so the warp only stages
      } else if (paired) {
        // two 4-channel groups (channels cg..cg+7) into every accumulator
        auto pair8 = [&](int cg) {
#pragma unroll
          for (int i = 0; i < DPW; ++i) {
            const uint32_t* const e = sa + ((warp * DPW + i) << cc_log) + cg;
            const uint4 a4 = *reinterpret_cast<const uint4*>(e);
            const uint4 b4 = *reinterpret_cast<const uint4*>(e + 4);
            const uint32_t q0 = a4.x + lane_off, q1 = a4.y + lane_off;
            const uint32_t q2 = a4.z + lane_off, q3 = a4.w + lane_off;
            const uint32_t q4 = b4.x + lane_off, q5 = b4.y + lane_off;
            const uint32_t q6 = b4.z + lane_off, q7 = b4.w + lane_off;
#pragma unroll
            for (int j = 0; j < K; ++j) {
              if constexpr (FMT == FMT_NIB)
                acc[i][j].add8_flush(lds32(q0 + 128u * j), lds32(q1 + 128u * j),
                                     lds32(q2 + 128u * j), lds32(q3 + 128u * j),
                                     lds32(q4 + 128u * j), lds32(q5 + 128u * j),
                                     lds32(q6 + 128u * j), lds32(q7 + 128u * j));
              if constexpr (FMT == FMT_TRI)
                acc[i][j].add8(lds32(q0 + 128u * j), lds32(q1 + 128u * j),
                               lds32(q2 + 128u * j), lds32(q3 + 128u * j),
                               lds32(q4 + 128u * j), lds32(q5 + 128u * j),
                               lds32(q6 + 128u * j), lds32(q7 + 128u * j));
            }
          }
        };
        if constexpr (FMT == FMT_NIB) {
          // 2-bit input: pairs of 4-channel groups widened together; a pair
          // adds at most two group sums to a byte lane, so byte lanes take
          // f1/2 pairs between 16-bit flushes.  The flush is taken before a
          // chunk whose pairs would pass that, so the pair loop itself has
          // no branch.
          const int npairs = cc >> 3;
          if (g1 + npairs > (p.f1 >> 1)) {
            g1 = 0;
#pragma unroll
            for (int i = 0; i < DPW; ++i)
#pragma unroll
              for (int j = 0; j < K; ++j) {
                acc[i][j].pair_fix();
                acc[i][j].flush1();
              }
            if (WIDE && ++g2 == p.f2) {
              g2 = 0;
#pragma unroll
              for (int i = 0; i < DPW; ++i)
#pragma unroll
                for (int j = 0; j < K; ++j) acc[i][j].flush2();
            }
          }
          g1 += npairs;
          for (int cg = 0; cg < cc; cg += 8) pair8(cg);
        }
        if constexpr (FMT == FMT_TRI) {
          // 8-bit input in 10-bit lanes: lane 2 of the separated sums holds
          // two pairs, then moves to its 32-bit sum
          for (int cg = 0; cg < cc; cg += 16) {
            pair8(cg);
            if (cc > 8) pair8(cg + 8);
#pragma unroll
            for (int i = 0; i < DPW; ++i)
#pragma unroll
              for (int j = 0; j < K; ++j) acc[i][j].flush1();
          }
        }
      } else
      for (int cg = 0; cg < cc; cg += 4) {
#pragma unroll
        for (int i = 0; i < DPW; ++i) {
          const uint4 a4 = *reinterpret_cast<const uint4*>(sa + ((warp * DPW + i) << cc_log) + cg);
          const uint32_t q0 = a4.x + lane_off, q1 = a4.y + lane_off;
          const uint32_t q2 = a4.z + lane_off, q3 = a4.w + lane_off;
#pragma unroll
          for (int j = 0; j < K; ++j)
            acc[i][j].add4(lds32(q0 + 128u * j), lds32(q1 + 128u * j), lds32(q2 + 128u * j),
                           lds32(q3 + 128u * j));
        }
        if (++g0 == p.f0) {
          g0 = 0;
#pragma unroll
          for (int i = 0; i < DPW; ++i)
#pragma unroll
            for (int j = 0; j < K; ++j) acc[i][j].flush0();
          if (++g1 == p.f1) {
            g1 = 0;
#pragma unroll
            for (int i = 0; i < DPW; ++i)
#pragma unroll
              for (int j = 0; j < K; ++j) acc[i][j].flush1();
            if (WIDE && ++g2 == p.f2) {
              g2 = 0;
#pragma unroll
              for (int i = 0; i < DPW; ++i)
#pragma unroll
                for (int j = 0; j < K; ++j) acc[i][j].flush2();
            }
          }
        }
      }
    }
    if constexpr (FMT == FMT_NIB) {
      if (paired) {
#pragma unroll
        for (int i = 0; i < DPW; ++i)
#pragma unroll
          for (int j = 0; j < K; ++j) acc[i][j].pair_fix();
      }
    }
    // all warps are done with this item's buffers before the next prologue
    __syncthreads();

    // (d) exact sums out: u32 rows, float rows, or 16-bit image rows
#pragma unroll
    for (int i = 0; i < DPW; ++i) {
      const int slot = warp * DPW + i;
      if (slot >= nd) continue;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        uint32_t v[SPW];
        acc[i][j].final(v);
        const int64_t tw = t0 + (int64_t)SPW * (lane + 32 * j);
        if (OUTK == OUT_HALFIMG) {
          uint32_t* dst = out_g + (int64_t)(d0 + slot) * S.out_stride + (tw >> 1);
          if (SPW == 8) {
            *reinterpret_cast<uint4*>(dst) =
                make_uint4(v[0] | (v[1 % SPW] << 16), v[2 % SPW] | (v[3 % SPW] << 16),
                           v[4 % SPW] | (v[5 % SPW] << 16), v[6 % SPW] | (v[7 % SPW] << 16));
          } else if (SPW == 4) {
            *reinterpret_cast<uint2*>(dst) =
                make_uint2(v[0] | (v[1 % SPW] << 16), v[2 % SPW] | (v[3 % SPW] << 16));
          } else if (SPW == 2) {
            dst[0] = v[0] | (v[1 % SPW] << 16);
          }
        } else if (OUTK == OUT_NARROW) {
          // scaled low-bit output: the top out_bits of the sum's range
          const uint32_t cap = (1u << p.out_bits) - 1u;
          uint32_t w[SPW];
#pragma unroll
          for (int e = 0; e < SPW; ++e) w[e] = min(v[e] >> p.out_shift, cap);
          const int esz = p.out_bits >> 3;
          char* const row = reinterpret_cast<char*>(S.out) +
                            ((int64_t)grp * S.g_out + (int64_t)(d0 + slot) * S.out_stride + tw) *
                                esz;
          const bool full = p.vec_out && tw + SPW <= t_end;
          if (esz == 2 && full && (SPW == 2 || SPW == 4 || SPW == 8)) {
            uint32_t u[SPW / 2 > 0 ? SPW / 2 : 1];
#pragma unroll
            for (int q = 0; q < SPW / 2; ++q) u[q] = w[2 * q] | (w[(2 * q + 1) % SPW] << 16);
            if (SPW == 8)
              *reinterpret_cast<uint4*>(row) = make_uint4(u[0], u[1 % (SPW / 2)],
                                                          u[2 % (SPW / 2)], u[3 % (SPW / 2)]);
            else if (SPW == 4)
              *reinterpret_cast<uint2*>(row) = make_uint2(u[0], u[1 % (SPW / 2)]);
            else
              *reinterpret_cast<uint32_t*>(row) = u[0];
          } else if (esz == 1 && full && (SPW == 4 || SPW == 8)) {
            uint32_t u[SPW / 4 > 0 ? SPW / 4 : 1];
#pragma unroll
            for (int q = 0; q < SPW / 4; ++q)
              u[q] = w[4 * q] | (w[(4 * q + 1) % SPW] << 8) | (w[(4 * q + 2) % SPW] << 16) |
                     (w[(4 * q + 3) % SPW] << 24);
            if (SPW == 8)
              *reinterpret_cast<uint2*>(row) = make_uint2(u[0], u[1 % (SPW / 4)]);
            else
              *reinterpret_cast<uint32_t*>(row) = u[0];
          } else if (esz == 2) {
#pragma unroll
            for (int e = 0; e < SPW; ++e)
              if (tw + e < t_end) reinterpret_cast<uint16_t*>(row)[e] = (uint16_t)w[e];
          } else {
#pragma unroll
            for (int e = 0; e < SPW; ++e)
              if (tw + e < t_end) reinterpret_cast<uint8_t*>(row)[e] = (uint8_t)w[e];
          }
        } else {
          uint32_t* dst = out_g + (int64_t)(d0 + slot) * S.out_stride + tw;
          if (p.vec_out && SPW >= 4 && tw + SPW <= t_end) {
#pragma unroll
            for (int q = 0; q < SPW / 4; ++q)
              reinterpret_cast<uint4*>(dst)[q] =
                  make_uint4(v[(4 * q) % SPW], v[(4 * q + 1) % SPW], v[(4 * q + 2) % SPW],
                             v[(4 * q + 3) % SPW]);
          } else if (p.vec_out && SPW == 2 && tw + 2 <= t_end) {
            *reinterpret_cast<uint2*>(dst) = make_uint2(v[0], v[1 % SPW]);
          } else {
#pragma unroll
            for (int e = 0; e < SPW; ++e)
              if (tw + e < t_end) dst[e] = v[e];
          }
        }
      }
    }
  }
}

// Host helpers used by the per-format translation units.
template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG>
cudaError_t launch_one(const LaunchParams& p, int grid, size_t smem, cudaStream_t st) {
  auto kern = k_dedisp<FMT, OUTK, WIDE, NWARP, DPW, K, PBG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NWARP * 32, smem, st>>>(p);
  return cudaGetLastError();
}

template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG>
cudaError_t occupancy_one(size_t smem, int* nblk) {
  auto kern = k_dedisp<FMT, OUTK, WIDE, NWARP, DPW, K, PBG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nblk, kern, NWARP * 32, smem);
}

template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG>
cudaError_t run_one(const LaunchParams* p, int grid, size_t smem, cudaStream_t st, int* occ) {
  return occ ? occupancy_one<FMT, OUTK, WIDE, NWARP, DPW, K, PBG>(smem, occ)
             : launch_one<FMT, OUTK, WIDE, NWARP, DPW, K, PBG>(*p, grid, smem, st);
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
