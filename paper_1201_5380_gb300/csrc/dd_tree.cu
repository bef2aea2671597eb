// The piecewise linear tree method (Sec. 3.1.1) for sm_103a.
//
// Stage 1 (Eq. subband_result): the basic tree of Sec. 3.1 on every sub-band
// of N' channels.  The tree needs log2 N' dependent steps over the whole
// block of channels; the paper ran one kernel per step through global memory
// because its GPUs could not hold a block in shared memory (Sec. 3.3).  Here
// one thread block owns one sub-band x one time tile: it unpacks the packed
// input rows of the sub-band straight into shared memory (T + N' - 1 samples
// per channel: the tree's total delay across N' channels is N' - 1), runs
// every step there between two buffers, and writes only the trails stage 2
// reads (d' up to the largest d'_n(d) of the sub-band).  Samples are 16-bit
// lanes, two per 32-bit word, so one add serves two samples: a sub-band's
// sums (N' * max sample) stay below 2^16.  Where they stay below 256 the
// trails are written in 8-bit lanes, four samples a word, and stage 2 reads
// half the words.
//
// Step i (radix r = 2^i), Eq. (tree_algorithm_first .. last):
//   A'[2v + j][t] = A[Phi(r, 2v)][t] + A[Phi(r, 2v + 1)][t + Theta(i, 2v + j)]
// with Theta of Eq. (tree_integer_delay) and the shuffle Phi of Eq.
// (shuffle); after the last step row d' holds trail d'.
//
// Stage 2 (Eq. combining_subbands): D[d][t] = sum_n S[n][d'_n(d)][t + dt''_n(d)]
// with d'_n(d) = delay(d, nu_{n+1}) - delay(d, nu_n) and dt''_n(d) =
// delay(d, nu_n) (the telescoped sum), from host-built per-trial tables.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "dd_internal.h"

namespace dd {
namespace {

// Output samples per stage-1 block: the two shared buffers of N' rows x
// (T + N') / 2 words stay near 35 KB each, so several blocks share an SM.
__host__ __device__ constexpr int tree_tile(int nsub) { return nsub <= 32 ? 512 : (nsub == 64 ? 256 : 128); }
__host__ __device__ constexpr int tree_words(int nsub) { return ((tree_tile(nsub) + nsub) / 2) | 1; }
// Row pitch: the WW loaded words, then zero words that the shifted reads of
// the last words run into (a pass reads at most 3 N'/8 + 3 words ahead), odd.
__host__ __device__ constexpr int tree_pitch(int nsub) { return (tree_words(nsub) + nsub / 2 + 4) | 1; }
constexpr int kTreeThreads = 512;
constexpr int kMaxTreeChans = 128;

struct TreeS1 {
  const uint8_t* in;      // packed time-major rows
  int64_t in_stride;      // bytes per row
  int64_t in_rows;        // valid rows (zeros beyond)
  const uint8_t* mask;    // nchans, 0 = killed
  uint32_t* S;            // stage-1 rows: two 16-bit or (OUT8) four 8-bit samples a word
  int64_t s_pitch;        // words per S row
  const int32_t* roff;    // first S row of each sub-band (+ end)
  int nbits;
  int nsb;                // sub-bands
};

// Eq. (shuffle) and Eq. (tree_integer_delay), truncated divisions.
__device__ __forceinline__ int tree_phi(int r, int v) { return (v & 1) * r + v / 2 + (v / (2 * r)) * r; }
__device__ __forceinline__ int tree_theta(int r, int v) { return ((v & (2 * r - 1)) + 1) >> 1; }

// Where the last pass writes: stage-1 rows r0 .. r0 + nrow - 1 (the trails
// 0 .. nrow - 1 of the sub-band), words of this tile from S.
struct TreeOut {
  uint32_t* S;
  int64_t s_pitch;
  int r0, nrow;
};

// Words of a row shifted by an odd sample: the high half of w0 and the low
// half of w1 (two 16-bit samples per word, earlier sample low).
__device__ __forceinline__ uint32_t half_shift(uint32_t w0, uint32_t w1) {
  return __funnelshift_r(w0, w1, 16);
}

// Two steps of the tree at once, steps i and i + 1 (radix R = 2^i): in each
// block of 4R rows, output K = 4m + sub takes trail m of its four quarters
// j = 0..3, quarter j shifted by j*m plus 0, sub/2, (sub+1)/2, sub samples
// (j = 0, 1, 2, 3): the composition of the two steps' Theta and Phi.
// Word q of outputs 4g .. 4g + 3 (g = sb * R + m) into r.
template <int NSUB, int R>
__device__ __forceinline__ void radix4_words(const uint32_t* src, int sb, int m, int q,
                                             uint32_t (&r)[4]) {
  constexpr int PW = tree_pitch(NSUB);
  const uint32_t* q0 = src + ((4 * sb + 0) * R + m) * PW + q;
  const uint32_t* q1 = src + ((4 * sb + 1) * R + m) * PW + q + (m >> 1);
  const uint32_t* q2 = src + ((4 * sb + 2) * R + m) * PW + q + m;
  const uint32_t* q3 = src + ((4 * sb + 3) * R + m) * PW + q + ((3 * m) >> 1);
  const int ps = (m & 1) * 16;  // quarters 1 and 3 start on an odd sample when m is odd
  const uint32_t a = q0[0];
  const uint32_t b0 = __funnelshift_r(q1[0], q1[1], ps), b1 = __funnelshift_r(q1[1], q1[2], ps);
  const uint32_t c0 = q2[0], c1 = q2[1];
  const uint32_t d0 = __funnelshift_r(q3[0], q3[1], ps), d1 = __funnelshift_r(q3[1], q3[2], ps);
  const uint32_t d2 = __funnelshift_r(q3[2], q3[3], ps);
  const uint32_t b_1 = half_shift(b0, b1), c_1 = half_shift(c0, c1);
  r[0] = a + b0 + c0 + d0;
  r[1] = a + b0 + c_1 + half_shift(d0, d1);
  r[2] = a + b_1 + c_1 + d1;
  r[3] = a + b_1 + c1 + half_shift(d1, d2);
}

// The last pass of a tile writes the trails to global memory: as 16-bit
// lanes (one word of the pass per word), or (OUT8) as 8-bit lanes, four
// samples a word made of two adjacent words of the pass by one byte
// permute (bytes 0 and 2 of each: the sums are below 128).
__device__ __forceinline__ uint32_t pack_bytes(uint32_t lo, uint32_t hi) {
  return __byte_perm(lo, hi, 0x6420u);
}

template <int NSUB, int R, bool LAST, bool OUT8>
__device__ __forceinline__ void tree_radix4(const uint32_t* src, uint32_t* dst, const TreeOut& o) {
  constexpr int T = tree_tile(NSUB), WW = tree_words(NSUB), PW = tree_pitch(NSUB);
  if constexpr (LAST && OUT8) {
    constexpr int QN = T / 4;
    for (int e = threadIdx.x; e < (NSUB / 4) * QN; e += kTreeThreads) {
      const int g = e / QN;
      const int q = e - g * QN;
      const int o0 = 4 * g;
      if (o0 >= o.nrow) continue;
      uint32_t ra[4], rb[4];
      radix4_words<NSUB, R>(src, g / R, g % R, 2 * q, ra);
      radix4_words<NSUB, R>(src, g / R, g % R, 2 * q + 1, rb);
#pragma unroll
      for (int sub = 0; sub < 4; ++sub)
        if (o0 + sub < o.nrow)
          o.S[(int64_t)(o.r0 + o0 + sub) * o.s_pitch + q] = pack_bytes(ra[sub], rb[sub]);
    }
  } else {
    constexpr int QN = LAST ? T / 2 : WW;  // the last pass writes only the tile
    for (int e = threadIdx.x; e < (NSUB / 4) * QN; e += kTreeThreads) {
      const int g = e / QN;
      const int q = e - g * QN;
      const int o0 = 4 * g;
      if (LAST && o0 >= o.nrow) continue;
      uint32_t r[4];
      radix4_words<NSUB, R>(src, g / R, g % R, q, r);
#pragma unroll
      for (int sub = 0; sub < 4; ++sub) {
        if (LAST) {
          if (o0 + sub < o.nrow) o.S[(int64_t)(o.r0 + o0 + sub) * o.s_pitch + q] = r[sub];
        } else {
          dst[(o0 + sub) * PW + q] = r[sub];
        }
      }
    }
  }
}

// One step (radix R = 2^i): outputs 2v and 2v + 1 take row lo and row hi = lo
// + R of their block of 2R rows, hi shifted by s = v mod R and s + 1
// samples (Theta of Eq. tree_integer_delay; lo and hi are Phi of Eq. shuffle).
// Word q of outputs 2v and 2v + 1 into r0, r1.
template <int NSUB, int R>
__device__ __forceinline__ void radix2_words(const uint32_t* src, int v, int q, uint32_t& r0,
                                             uint32_t& r1) {
  constexpr int PW = tree_pitch(NSUB);
  const int lo = tree_phi(R, 2 * v), hi = tree_phi(R, 2 * v + 1);
  const int sft = tree_theta(R, 2 * v);  // output 2v + 1: sft + 1
  const uint32_t a = src[lo * PW + q];
  const uint32_t* h = src + hi * PW + q + (sft >> 1);
  const int ps = (sft & 1) * 16;
  const uint32_t h0 = __funnelshift_r(h[0], h[1], ps), h1 = __funnelshift_r(h[1], h[2], ps);
  r0 = a + h0;
  r1 = a + half_shift(h0, h1);
}

template <int NSUB, int R, bool LAST, bool OUT8>
__device__ __forceinline__ void tree_radix2(const uint32_t* src, uint32_t* dst, const TreeOut& o) {
  constexpr int T = tree_tile(NSUB), WW = tree_words(NSUB), PW = tree_pitch(NSUB);
  if constexpr (LAST && OUT8) {
    constexpr int QN = T / 4;
    for (int e = threadIdx.x; e < (NSUB / 2) * QN; e += kTreeThreads) {
      const int v = e / QN;
      const int q = e - v * QN;
      const int o0 = 2 * v;
      if (o0 >= o.nrow) continue;
      uint32_t a0, a1, b0, b1;
      radix2_words<NSUB, R>(src, v, 2 * q, a0, a1);
      radix2_words<NSUB, R>(src, v, 2 * q + 1, b0, b1);
      o.S[(int64_t)(o.r0 + o0) * o.s_pitch + q] = pack_bytes(a0, b0);
      if (o0 + 1 < o.nrow) o.S[(int64_t)(o.r0 + o0 + 1) * o.s_pitch + q] = pack_bytes(a1, b1);
    }
  } else {
    constexpr int QN = LAST ? T / 2 : WW;
    for (int e = threadIdx.x; e < (NSUB / 2) * QN; e += kTreeThreads) {
      const int v = e / QN;
      const int q = e - v * QN;
      const int o0 = 2 * v;
      if (LAST && o0 >= o.nrow) continue;
      uint32_t r0, r1;
      radix2_words<NSUB, R>(src, v, q, r0, r1);
      if (LAST) {
        o.S[(int64_t)(o.r0 + o0) * o.s_pitch + q] = r0;
        if (o0 + 1 < o.nrow) o.S[(int64_t)(o.r0 + o0 + 1) * o.s_pitch + q] = r1;
      } else {
        dst[o0 * PW + q] = r0;
        dst[(o0 + 1) * PW + q] = r1;
      }
    }
  }
}

// Steps I .. log2 N' - 1, reading src and writing dst (buffers alternate).
template <int NSUB, int I, bool OUT8>
__device__ __forceinline__ void tree_passes(uint32_t* src, uint32_t* dst, const TreeOut& o) {
  constexpr int M = (NSUB >= 2) + (NSUB >= 4) + (NSUB >= 8) + (NSUB >= 16) + (NSUB >= 32) +
                    (NSUB >= 64) + (NSUB >= 128);  // log2 N'
  if constexpr (I + 1 < M) {
    tree_radix4<NSUB, (1 << I), I + 2 == M, OUT8>(src, dst, o);
    if constexpr (I + 2 < M) {
      __syncthreads();
      tree_passes<NSUB, I + 2, OUT8>(dst, src, o);
    }
  } else if constexpr (I < M) {
    tree_radix2<NSUB, (1 << I), true, OUT8>(src, dst, o);
  }
}

template <int NSUB, bool OUT8>
__global__ void __launch_bounds__(kTreeThreads) k_tree_stage1(const TreeS1 p) {
  constexpr int T = tree_tile(NSUB);
  constexpr int WW = tree_words(NSUB);
  constexpr int PW = tree_pitch(NSUB);
  constexpr int NWARP = kTreeThreads / 32;
  extern __shared__ uint32_t sm[];
  uint32_t* buf0 = sm;
  uint32_t* buf1 = sm + NSUB * PW;
  // blocks in order (tile, sub-band), sub-band fastest: the blocks running
  // together read whole input rows between them
  const int n = (int)(blockIdx.x % p.nsb);
  const int64_t t0 = (int64_t)(blockIdx.x / p.nsb) * T;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int nb = p.nbits;
  const uint32_t vmask = (1u << nb) - 1u;

  // (a) unpack: a thread takes two consecutive rows (time samples) of the
  //     sub-band at a time and writes each channel's pair of samples as one
  //     word of that channel's row (16-bit lanes, earlier sample low)
  {
    const int64_t bit0 = (int64_t)n * NSUB * nb;  // a multiple of 8 unless N'*nbits < 8
    const int sub_bits = NSUB * nb;
    const bool words = (sub_bits % 32) == 0 &&
                       ((reinterpret_cast<uintptr_t>(p.in) | (uintptr_t)p.in_stride |
                         (uintptr_t)(bit0 >> 3)) & 3) == 0;
    if (words) {
      // one (word of the tile, 32-bit piece of the sub-band's bits) per
      // thread, so that every thread has a share
      const int nw = sub_bits / 32;
      for (int e = tid; e < WW * nw; e += kTreeThreads) {
        const int q = e / nw, w = e - q * nw;
        const int64_t t = t0 + 2 * q;
        const uint8_t* r0 = p.in + t * p.in_stride + (bit0 >> 3);
        const uint8_t* r1 = r0 + p.in_stride;
        const uint32_t x0 = t < p.in_rows ? __ldg(reinterpret_cast<const uint32_t*>(r0) + w) : 0u;
        const uint32_t x1 =
            t + 1 < p.in_rows ? __ldg(reinterpret_cast<const uint32_t*>(r1) + w) : 0u;
        for (int j = 0; j < 32 / nb; ++j) {
          const int c = w * (32 / nb) + j;
          buf0[c * PW + q] = ((x0 >> (j * nb)) & vmask) | (((x1 >> (j * nb)) & vmask) << 16);
        }
      }
    } else {
      const int sh = (int)(bit0 & 7);
      for (int q = tid; q < WW; q += kTreeThreads) {
        const int64_t t = t0 + 2 * q;
        const uint8_t* r0 = p.in + t * p.in_stride + (bit0 >> 3);
        const uint8_t* r1 = r0 + p.in_stride;
        const bool ok0 = t < p.in_rows, ok1 = t + 1 < p.in_rows;
        for (int c = 0; c < NSUB; ++c) {
          const int b = sh + c * nb;
          const uint32_t x0 = ok0 ? ((uint32_t)__ldg(r0 + (b >> 3)) >> (b & 7)) & vmask : 0u;
          const uint32_t x1 = ok1 ? ((uint32_t)__ldg(r1 + (b >> 3)) >> (b & 7)) & vmask : 0u;
          buf0[c * PW + q] = x0 | (x1 << 16);
        }
      }
    }
    // the zero words past each row, in both buffers (never written again)
    for (int e = tid; e < 2 * NSUB * (PW - WW); e += kTreeThreads) {
      const int row = e / (PW - WW);
      sm[row * PW + WW + (e - row * (PW - WW))] = 0u;
    }
    __syncthreads();
    // the kill mask: a killed channel's row reads zero
    for (int c = warp; c < NSUB; c += NWARP)
      if (!__ldg(p.mask + n * NSUB + c))
        for (int q = lane; q < WW; q += 32) buf0[c * PW + q] = 0u;
  }
  __syncthreads();

  // (b) the log2 N' steps, two at a time where it can (a radix-4 pass), out
  //     of place between the two buffers; the last pass writes the trails
  //     stage 2 reads straight to global memory
  TreeOut o;
  o.r0 = __ldg(p.roff + n);
  o.nrow = __ldg(p.roff + n + 1) - o.r0;
  o.S = p.S + t0 / (OUT8 ? 4 : 2);
  o.s_pitch = p.s_pitch;
  tree_passes<NSUB, 0, OUT8>(buf0, buf1, o);
}

struct TreeS2 {
  const uint32_t* S;      // stage-1 rows: two 16-bit (or four 8-bit) samples a word
  int64_t s_pitch;        // words per S row
  const int2* tab;        // [trial][sub-band] {S row, shift}
  int nsb, ndm;
  int flush;              // sub-bands a 16-bit lane sum takes before widening
  int vec_out;            // rows 8-byte aligned: pairs of samples stored at once
  int64_t nsamps;
  uint32_t* out;
  int64_t out_stride;
};

constexpr int kS2Warps = 8;  // trials per block
constexpr int kS2W = 8;      // words per lane (two samples each, stride 32 words)
constexpr int kS2Tile = 64 * kS2W;  // samples per warp
// S words stage 2 may read past the last sample it uses (whole words of the
// last tile, and the word after them): the allocation carries them
constexpr int64_t kS2SlackWords = 32 * kS2W + 64;

// A warp sums one trial over a tile of 512 samples: lane l holds samples
// 2(l + 32j) and 2(l + 32j) + 1 of the tile (j < 8) in one word, two 16-bit
// lanes.  A sub-band's shifted row is read a word per lane and sample pair;
// an odd shift takes the word after each lane's from the next lane (a warp
// shuffle; lane 31 from lane 0's next word) and funnel-shifts the pair into
// place, so every load is an aligned, coalesced 32-bit load.  The next
// sub-band's words are loaded while this one's are summed (the kernel is
// bound by the loads in flight).  WIDEN: the 16-bit sums are widened into
// 32-bit sums every p.flush sub-bands (the host's bound: flush * N' * max
// sample < 2^16); otherwise only at the end.
template <bool WIDEN>
__global__ void __launch_bounds__(kS2Warps * 32, 5) k_tree_stage2(const TreeS2 p) {
  extern __shared__ int2 s_tab[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // blocks in order (time tile, trial block), trial block fastest: the
  // blocks running together read the same stage-1 tiles, from L2
  const int ntb = (p.ndm + kS2Warps - 1) / kS2Warps;
  const int d0 = (int)(blockIdx.x % ntb) * kS2Warps;
  const int64_t t0 = (int64_t)(blockIdx.x / ntb) * kS2Tile;
  const int nd = min(kS2Warps, p.ndm - d0);
  for (int e = threadIdx.x; e < nd * p.nsb; e += blockDim.x)
    s_tab[e] = p.tab[(int64_t)d0 * p.nsb + e];
  __syncthreads();
  if (warp >= nd) return;
  const int d = d0 + warp;
  const int2* tab = s_tab + warp * p.nsb;
  uint32_t h[kS2W], u[WIDEN ? 2 * kS2W : 1];
#pragma unroll
  for (int j = 0; j < kS2W; ++j) h[j] = 0u;
#pragma unroll
  for (int j = 0; j < (WIDEN ? 2 * kS2W : 1); ++j) u[j] = 0u;

  // words of sub-band n (and lane 0's word after them); returns the shift's
  // parity
  auto fetch = [&](int n, uint32_t (&w)[kS2W], uint32_t& tail) -> bool {
    const int2 rs = tab[n];
    const int64_t e0 = t0 + rs.y;  // sample of the row under the tile's first output
    const uint32_t* src = p.S + (int64_t)rs.x * p.s_pitch + (e0 >> 1) + lane;
#pragma unroll
    for (int j = 0; j < kS2W; ++j) w[j] = __ldg(src + 32 * j);
    tail = lane == 0 ? __ldg(src + 32 * kS2W) : 0u;
    return (e0 & 1) != 0;
  };
  auto accumulate = [&](const uint32_t (&w)[kS2W], uint32_t tail, bool odd) {
    if (odd) {
#pragma unroll
      for (int j = 0; j < kS2W; ++j) {
        // lanes 1..31 send their word j, lane 0 its next one (for lane 31)
        const uint32_t give = lane == 0 ? (j + 1 < kS2W ? w[(j + 1) % kS2W] : tail) : w[j];
        const uint32_t nx = __shfl_sync(0xffffffffu, give, (lane + 1) & 31);
        h[j] += __funnelshift_r(w[j], nx, 16);
      }
    } else {
#pragma unroll
      for (int j = 0; j < kS2W; ++j) h[j] += w[j];
    }
  };
  auto widen = [&]() {
    if constexpr (WIDEN) {
#pragma unroll
      for (int j = 0; j < kS2W; ++j) {
        u[2 * j] += h[j] & 0xFFFFu;
        u[2 * j + 1] += h[j] >> 16;
        h[j] = 0u;
      }
    }
  };

  uint32_t wa[kS2W], wb[kS2W], ta, tb;
  bool oa = fetch(0, wa, ta);
  int g = 0;
  for (int n = 0; n < p.nsb; n += 2) {
    // sub-bands n (in wa) and n + 1 (in wb); the loads of the next one are
    // in flight while each is summed
    const bool two = n + 1 < p.nsb;
    bool ob = false;
    if (two) ob = fetch(n + 1, wb, tb);
    accumulate(wa, ta, oa);
    if (WIDEN && ++g == p.flush) {
      g = 0;
      widen();
    }
    if (!two) break;
    if (n + 2 < p.nsb) oa = fetch(n + 2, wa, ta);
    accumulate(wb, tb, ob);
    if (WIDEN && ++g == p.flush) {
      g = 0;
      widen();
    }
  }
  uint32_t v[2 * kS2W];
  if constexpr (WIDEN) {
    widen();
#pragma unroll
    for (int j = 0; j < 2 * kS2W; ++j) v[j] = u[WIDEN ? j : 0];
  } else {
#pragma unroll
    for (int j = 0; j < kS2W; ++j) {
      v[2 * j] = h[j] & 0xFFFFu;
      v[2 * j + 1] = h[j] >> 16;
    }
  }
  uint32_t* o = p.out + (int64_t)d * p.out_stride;
#pragma unroll
  for (int j = 0; j < kS2W; ++j) {
    const int64_t t = t0 + 2 * (lane + 32 * j);
    if (p.vec_out && t + 2 <= p.nsamps) {
      *reinterpret_cast<uint2*>(o + t) = make_uint2(v[2 * j], v[2 * j + 1]);
    } else {
      if (t < p.nsamps) o[t] = v[2 * j];
      if (t + 1 < p.nsamps) o[t + 1] = v[2 * j + 1];
    }
  }
}

// Stage 2 over 8-bit trails (four samples a word): the same per-trial sum
// over sub-bands, half the loads.  A lane's words are shifted by the trial's
// sample offset mod 4 (one byte a sample) with the next word taken from the
// neighbouring lane, as above; then (PAIRS: trails below 128) two sub-bands
// are added in each byte lane without a carry, or (trails below 256) each
// sub-band is taken alone, and spread into 16-bit sums, samples {0, 2} by a
// mask and {1, 3} by a byte permute.  The host takes this kernel only where
// a trial's total fits 16 bits.
constexpr int kS2W8 = kS2Tile / 128;  // words per lane (four samples each, stride 32 words)

template <bool PAIRS>
__global__ void __launch_bounds__(kS2Warps * 32, 5) k_tree_stage2_b8(const TreeS2 p) {
  extern __shared__ int2 s_tab[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ntb = (p.ndm + kS2Warps - 1) / kS2Warps;
  const int d0 = (int)(blockIdx.x % ntb) * kS2Warps;
  const int64_t t0 = (int64_t)(blockIdx.x / ntb) * kS2Tile;
  const int nd = min(kS2Warps, p.ndm - d0);
  for (int e = threadIdx.x; e < nd * p.nsb; e += blockDim.x)
    s_tab[e] = p.tab[(int64_t)d0 * p.nsb + e];
  __syncthreads();
  if (warp >= nd) return;
  const int d = d0 + warp;
  const int2* tab = s_tab + warp * p.nsb;
  uint32_t ev[kS2W8], od[kS2W8];
#pragma unroll
  for (int j = 0; j < kS2W8; ++j) ev[j] = od[j] = 0u;

  // words of sub-band n (and lane 0's word after them); returns the shift
  auto fetch = [&](int n, uint32_t (&w)[kS2W8], uint32_t& tail) -> int {
    const int2 rs = tab[n];
    const int64_t e0 = t0 + rs.y;
    const uint32_t* src = p.S + (int64_t)rs.x * p.s_pitch + (e0 >> 2) + lane;
#pragma unroll
    for (int j = 0; j < kS2W8; ++j) w[j] = __ldg(src + 32 * j);
    tail = lane == 0 ? __ldg(src + 32 * kS2W8) : 0u;
    return (int)(e0 & 3);
  };
  // in place: word j of the lane moved on by r samples (r is the trial's,
  // the same for the whole warp)
  auto shift = [&](uint32_t (&w)[kS2W8], uint32_t tail, int r) {
    if (r == 0) return;
#pragma unroll
    for (int j = 0; j < kS2W8; ++j) {
      const uint32_t give = lane == 0 ? (j + 1 < kS2W8 ? w[(j + 1) % kS2W8] : tail) : w[j];
      const uint32_t nx = __shfl_sync(0xffffffffu, give, (lane + 1) & 31);
      w[j] = __funnelshift_r(w[j], nx, 8 * r);
    }
  };
  auto spread = [&](int j, uint32_t a) {
    ev[j] += a & 0x00FF00FFu;
    od[j] += __byte_perm(a, 0u, 0x4341u);
  };

  // sub-bands n and n + 1 summed from one pair of buffers while the loads of
  // n + 2 and n + 3 are in flight in the other (eight words a lane in
  // flight, as many as the 16-bit kernel's one sub-band ahead)
  auto sum_pair = [&](uint32_t (&x)[kS2W8], uint32_t tx, int rx, uint32_t (&y)[kS2W8],
                      uint32_t ty, int ry, bool two) {
    shift(x, tx, rx);
    if (two) {
      shift(y, ty, ry);
#pragma unroll
      for (int j = 0; j < kS2W8; ++j) {
        if (PAIRS) {
          spread(j, x[j] + y[j]);
        } else {
          spread(j, x[j]);
          spread(j, y[j]);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < kS2W8; ++j) spread(j, x[j]);
    }
  };
  uint32_t a0[kS2W8], a1[kS2W8], b0[kS2W8], b1[kS2W8];
  uint32_t ta0 = 0u, ta1 = 0u, tb0 = 0u, tb1 = 0u;
  int ra0 = fetch(0, a0, ta0), ra1 = 0, rb0 = 0, rb1 = 0;
  if (p.nsb > 1) ra1 = fetch(1, a1, ta1);
  for (int n = 0;;) {
    if (n + 2 < p.nsb) rb0 = fetch(n + 2, b0, tb0);
    if (n + 3 < p.nsb) rb1 = fetch(n + 3, b1, tb1);
    sum_pair(a0, ta0, ra0, a1, ta1, ra1, n + 1 < p.nsb);
    if ((n += 2) >= p.nsb) break;
    if (n + 2 < p.nsb) ra0 = fetch(n + 2, a0, ta0);
    if (n + 3 < p.nsb) ra1 = fetch(n + 3, a1, ta1);
    sum_pair(b0, tb0, rb0, b1, tb1, rb1, n + 1 < p.nsb);
    if ((n += 2) >= p.nsb) break;
  }
  uint32_t* o = p.out + (int64_t)d * p.out_stride;
#pragma unroll
  for (int j = 0; j < kS2W8; ++j) {
    const uint32_t v[4] = {ev[j] & 0xFFFFu, od[j] & 0xFFFFu, ev[j] >> 16, od[j] >> 16};
    const int64_t t = t0 + 4 * (lane + 32 * j);
    if (p.vec_out && t + 4 <= p.nsamps) {
      *reinterpret_cast<uint2*>(o + t) = make_uint2(v[0], v[1]);
      *reinterpret_cast<uint2*>(o + t + 2) = make_uint2(v[2], v[3]);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (t + e < p.nsamps) o[t + e] = v[e];
    }
  }
}

template <int NSUB, bool OUT8>
cudaError_t launch_stage1(const TreeS1& a, int64_t tiles, int nsb, cudaStream_t st) {
  const size_t smem = 2u * NSUB * tree_pitch(NSUB) * 4u;
  auto k = k_tree_stage1<NSUB, OUT8>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)(tiles * nsb), kTreeThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// out8: 8-bit trails (N' * max sample < 256)
cudaError_t stage1(int nsub, bool out8, const TreeS1& a, int64_t tiles, int nsb,
                   cudaStream_t st) {
#define DD_TREE_CASE(N) \
  case N:               \
    return out8 ? launch_stage1<N, true>(a, tiles, nsb, st) : launch_stage1<N, false>(a, tiles, nsb, st);
  switch (nsub) {
    DD_TREE_CASE(2)
    DD_TREE_CASE(4)
    DD_TREE_CASE(8)
    DD_TREE_CASE(16)
    DD_TREE_CASE(32)
    DD_TREE_CASE(64)
    DD_TREE_CASE(128)
    default: return cudaErrorInvalidValue;
  }
#undef DD_TREE_CASE
}

}  // namespace

// Host tables of the piecewise linear tree: per trial and sub-band the
// stage-1 row (sub-band n's rows are its trails 0 .. max_d d'_n(d)) and the
// stage-2 shift.  d'_n(d) reads the delay at the band edge nu_{N_s} = N_nu
// for the last sub-band (Eq. 4 evaluated one channel past the band).
dd_status prepare_tree(Plan& p) {
  if (!p.tree_dirty) return DD_OK;
  const int Np = p.tree_chans;
  if (Np <= 0) return DD_ERR_INVALID_ARG;
  const int n = ndm(p), C = p.nchans, nsb = C / Np;
  const double dT_edge = partial_delay(p.f0, p.df, p.dt, C);
  std::vector<int32_t> dp((size_t)n * nsb), sh((size_t)n * nsb);
  std::vector<int32_t> dmax(nsb, 0);
  int32_t shmax = 0;
  for (int d = 0; d < n; ++d) {
    const int32_t* row = p.delays.data() + (size_t)d * C;
    const double edge = std::floor(p.dms[d] * dT_edge + 0.5);
    if (!(edge >= 0.0) || edge > 1.0e9) return DD_ERR_INVALID_ARG;
    for (int s = 0; s < nsb; ++s) {
      const int32_t a = row[(size_t)s * Np];
      const int32_t b = s + 1 < nsb ? row[(size_t)(s + 1) * Np] : (int32_t)edge;
      const int32_t v = b - a;
      if (v < 0 || v >= Np) return DD_ERR_INVALID_ARG;  // beyond the piecewise diagonal DM
      dp[(size_t)d * nsb + s] = v;
      sh[(size_t)d * nsb + s] = a;
      dmax[s] = std::max(dmax[s], v);
      shmax = std::max(shmax, a);
    }
  }
  p.tree_roff.assign(nsb + 1, 0);
  for (int s = 0; s < nsb; ++s) p.tree_roff[s + 1] = p.tree_roff[s] + dmax[s] + 1;
  p.tree_tab.resize((size_t)n * nsb * 2);
  for (int d = 0; d < n; ++d)
    for (int s = 0; s < nsb; ++s) {
      p.tree_tab[((size_t)d * nsb + s) * 2] = p.tree_roff[s] + dp[(size_t)d * nsb + s];
      p.tree_tab[((size_t)d * nsb + s) * 2 + 1] = sh[(size_t)d * nsb + s];
    }
  p.tree_shift_max = shmax;
  p.tree_dirty = false;
  p.tree_dev_dirty = true;
  return DD_OK;
}

// Input rows beyond the gulp: the largest stage-2 shift plus the tree's own
// reach, N' - 1 samples.
int64_t tree_input_extra(const Plan& p) { return (int64_t)p.tree_shift_max + p.tree_chans - 1; }

dd_status exec_tree(Plan& p, const ExecArgs& a) {
  if (a.in_nbits == 32) return DD_ERR_UNSUPPORTED_NBITS;
  dd_status s = prepare_tree(p);
  if (s != DD_OK) return s;
  const int Np = p.tree_chans, C = p.nchans, nsb = C / Np, n = ndm(p);
  cudaError_t e;
  if (p.tree_dev_dirty) {
    if ((e = p.d_tree_tab.ensure(p.tree_tab.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(p.d_tree_tab.p, p.tree_tab.data(), p.tree_tab.size() * 4,
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = p.d_tree_roff.ensure(p.tree_roff.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(p.d_tree_roff.p, p.tree_roff.data(), p.tree_roff.size() * 4,
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_status(e);
    p.tree_dev_dirty = false;
  }
  const int T = tree_tile(Np);
  const int64_t len1 = a.nsamps_out + p.tree_shift_max;  // S samples stage 2 reads
  const int64_t tiles = (len1 + T - 1) / T;
  // S rows: every stage-1 tile writes T samples; stage 2 reads up to len1
  const int64_t pitch = ((tiles * T + 63) / 64) * 64;    // samples
  const int rows = p.tree_roff[nsb];
  // 8-bit trails where a sub-band's sums stay below 256 and a trial's total
  // below 2^16, added two sub-bands a byte lane where they stay below 128;
  // else 16-bit
  const int64_t vmax = (1 << a.in_nbits) - 1;
  const bool b8 = Np * vmax <= 255 && C * vmax <= 65535;
  const bool pairs = Np * vmax <= 127;
  const int spw = b8 ? 4 : 2;
  if ((e = p.d_tree_S.ensure(((size_t)rows * pitch / spw + kS2SlackWords) * 4)) != cudaSuccess)
    return cuda_status(e);
  TreeS1 s1;
  s1.in = static_cast<const uint8_t*>(a.in);
  s1.in_stride = a.in_row_stride;
  s1.in_rows = a.in_rows;
  s1.mask = static_cast<const uint8_t*>(p.d_mask.p);
  s1.S = static_cast<uint32_t*>(p.d_tree_S.p);
  s1.s_pitch = pitch / spw;
  s1.roff = static_cast<const int32_t*>(p.d_tree_roff.p);
  s1.nbits = a.in_nbits;
  s1.nsb = nsb;
  {
    KernelTimer kt(&p, DD_KERNEL_DEDISP, a.st);
    if ((e = stage1(Np, b8, s1, tiles, nsb, a.st)) != cudaSuccess) return cuda_status(e);
  }
  TreeS2 s2;
  s2.S = static_cast<const uint32_t*>(p.d_tree_S.p);
  s2.s_pitch = pitch / spw;
  s2.tab = static_cast<const int2*>(p.d_tree_tab.p);
  s2.nsb = nsb;
  s2.ndm = n;
  // a stage-1 sample is at most N' * (2^nbits - 1) (<= 128 * 255 < 2^16)
  s2.flush = (int)(65535 / ((int64_t)Np * ((1 << a.in_nbits) - 1)));
  s2.vec_out = (reinterpret_cast<uintptr_t>(a.out) & 7) == 0 && (a.out_stride & 1) == 0;
  s2.nsamps = a.nsamps_out;
  s2.out = static_cast<uint32_t*>(a.out);
  s2.out_stride = a.out_stride;
  const int64_t t2 = (a.nsamps_out + kS2Tile - 1) / kS2Tile;
  const unsigned grid = (unsigned)(t2 * ((n + kS2Warps - 1) / kS2Warps));
  const size_t smem = (size_t)kS2Warps * nsb * sizeof(int2);
  KernelTimer kt(&p, DD_KERNEL_STAGE2, a.st);
  if (b8 && pairs)
    k_tree_stage2_b8<true><<<grid, kS2Warps * 32, smem, a.st>>>(s2);
  else if (b8)
    k_tree_stage2_b8<false><<<grid, kS2Warps * 32, smem, a.st>>>(s2);
  else if (s2.flush < nsb)
    k_tree_stage2<true><<<grid, kS2Warps * 32, smem, a.st>>>(s2);
  else
    k_tree_stage2<false><<<grid, kS2Warps * 32, smem, a.st>>>(s2);
  return cuda_status(cudaGetLastError());
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_plan_set_tree(dd_plan plan, int chans_per_subband) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DD_ERR_INVALID_ARG;
  const int Np = chans_per_subband;
  if (Np != 0) {
    if (Np < 2 || Np > kMaxTreeChans || (Np & (Np - 1)) || p->nchans % Np) return DD_ERR_INVALID_ARG;
    if (!(p->f0 + (double)p->nchans * p->df > 0.0)) return DD_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(p->mu);
  p->tree_chans = Np;
  p->tree_dirty = true;
  return DD_OK;
}

extern "C" dd_status dd_plan_get_tree_dm_limit(dd_plan plan, int chans_per_subband,
                                              double* dm_diag) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  const int Np = chans_per_subband;
  if (!p || !dm_diag || Np < 2 || Np > p->nchans || (Np & (Np - 1)) || p->nchans % Np)
    return DD_ERR_INVALID_ARG;
  if (!(p->f0 + (double)p->nchans * p->df > 0.0)) return DD_ERR_INVALID_ARG;
  const double hi = partial_delay(p->f0, p->df, p->dt, p->nchans);
  const double lo = partial_delay(p->f0, p->df, p->dt, p->nchans - Np);
  *dm_diag = ((double)Np - 0.5) / (hi - lo);
  return DD_OK;
}
