// Corner turn (unpack + transpose into the staged image), the integer-add
// probe, and the format dispatch of the dedispersion kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dd_internal.h"

namespace dd {

cudaError_t dispatch_nib(int, bool, int, bool, const LaunchParams*, int, size_t, cudaStream_t,
                         int*);
cudaError_t dispatch_byte(int, bool, int, bool, const LaunchParams*, int, size_t, cudaStream_t,
                          int*);
cudaError_t dispatch_half(int, bool, int, bool, const LaunchParams*, int, size_t, cudaStream_t,
                          int*);
cudaError_t dispatch_word(int, int, bool, int, bool, const LaunchParams*, int, size_t,
                          cudaStream_t, int*);
cudaError_t dispatch_tri(int, bool, int, bool, const LaunchParams*, int, size_t, cudaStream_t,
                         int*);
cudaError_t dispatch_nib_mt(int, bool, int, bool, const LaunchParams*, int, size_t, cudaStream_t,
                            int*);
cudaError_t dispatch_half_mt(int, bool, int, bool, const LaunchParams*, int, size_t,
                             cudaStream_t, int*);
cudaError_t dispatch_sb8_mt(int, bool, int, bool, const LaunchParams*, int, size_t,
                            cudaStream_t, int*);

bool multi_tile_compiled(int fmt, int outk, bool wide, int cfg) {
  if (fmt == FMT_NIB) return (outk == OUT_HALFIMG || outk == OUT_BYTEIMG) && !wide && cfg == 0;
  if (fmt == FMT_HALF) return cfg == 5 && ((outk == OUT_HALFIMG && !wide) || outk == OUT_U32);
  if (fmt == FMT_SB8) return cfg == 4 && outk == OUT_U32 && !wide;
  return false;
}

bool multi_tile_only(int fmt, int outk) { return fmt == FMT_SB8 || outk == OUT_BYTEIMG; }

static cudaError_t dispatch(int fmt, int outk, bool wide, int cfg, bool pbg, bool mt,
                            const LaunchParams* p, int grid, size_t smem, cudaStream_t st,
                            int* occ) {
  if (mt) {
    if (fmt == FMT_NIB) return dispatch_nib_mt(outk, wide, cfg, pbg, p, grid, smem, st, occ);
    if (fmt == FMT_HALF) return dispatch_half_mt(outk, wide, cfg, pbg, p, grid, smem, st, occ);
    if (fmt == FMT_SB8) return dispatch_sb8_mt(outk, wide, cfg, pbg, p, grid, smem, st, occ);
    return cudaErrorInvalidValue;
  }
  if (multi_tile_only(fmt, outk)) return cudaErrorInvalidValue;
  switch (fmt) {
    case FMT_NIB: return dispatch_nib(outk, wide, cfg, pbg, p, grid, smem, st, occ);
    case FMT_BYTE: return dispatch_byte(outk, wide, cfg, pbg, p, grid, smem, st, occ);
    case FMT_HALF: return dispatch_half(outk, wide, cfg, pbg, p, grid, smem, st, occ);
    case FMT_TRI: return dispatch_tri(outk, wide, cfg, pbg, p, grid, smem, st, occ);
    default: return dispatch_word(fmt, outk, wide, cfg, pbg, p, grid, smem, st, occ);
  }
}

cudaError_t launch_dedisp(int fmt, int outk, bool wide, int cfg, const LaunchParams& p,
                          int grid, size_t smem, cudaStream_t st) {
  return dispatch(fmt, outk, wide, cfg, p.per_block_geo != 0, p.multi_tile != 0, &p, grid, smem,
                  st, nullptr);
}

cudaError_t dedisp_max_blocks_per_sm(int fmt, int outk, bool wide, int cfg, bool pbg, bool mt,
                                     size_t smem, int* nblk) {
  *nblk = 0;
  return dispatch(fmt, outk, wide, cfg, pbg, mt, nullptr, 0, smem, nullptr, nblk);
}

// Two mbarriers, then two buffers each of the landing windows (cc x
// (nww+4), the unshifted copy) and the other SPW-1 shifted copies (cc x
// (SPW-1) x nww), then two address tables (B x cc).
size_t dedisp_smem_bytes(int fmt, int cfg, int cc, int nww) {
  const int B = kTileCfgs[cfg].nwarp * kTileCfgs[cfg].dpw;
  const size_t copies = (size_t)cc * (fmt_spw(fmt) - 1) * nww;
  const size_t landing = (size_t)cc * (nww + 4);
  return 16u + 4u * 2u * (landing + copies + (size_t)B * cc);
}

// ---------------------------------------------------------------------------
// Corner turn.  The paper transposes the input to frequency-major order by
// whole words before dedispersing (Sec. 2.3); here one pass unpacks the
// time-major 1/2/4/8-bit or float filterbank into per-channel image rows in
// the staged lane format, zeroes killed channels (the arithmetic kill mask
// of Sec. 2.3) and zero-pads outside [0, nrows_valid).
//
// Block = 256 threads over CB channels x WB image words.  Phase 1 reads the
// raw rows of the block (32 bytes per row for packed input, 128 for float)
// into shared memory with coalesced byte loads; phase 2 builds image words,
// consecutive threads writing consecutive words of one channel row.
// ---------------------------------------------------------------------------
template <int NBITS, int FMT>
__global__ void __launch_bounds__(256) k_corner_turn(const uint8_t* __restrict__ in,
                                                     int64_t in_stride, int64_t t_begin,
                                                     int64_t nrows_valid, int nchans,
                                                     const uint8_t* __restrict__ mask,
                                                     uint32_t* __restrict__ img,
                                                     int64_t row_words, int64_t w_first,
                                                     int64_t words) {
  constexpr bool F32 = (NBITS == 32);
  constexpr int SPW = FMT == FMT_TRI ? 3 : (F32 ? 1 : (NBITS <= 2 ? 8 : (NBITS == 4 ? 4 : 2)));
  constexpr int LW = FMT == FMT_TRI ? 10 : 32 / SPW;
  constexpr int ROWB = F32 ? 128 : 32;           // raw bytes per row in the block
  constexpr int CB = F32 ? 32 : 256 / NBITS;     // channels per block
  constexpr int WB = F32 ? 64 : 32;              // image words per block
  constexpr int R = WB * SPW;                    // raw rows per block
  constexpr int PITCH = ROWB + 4;
  __shared__ uint8_t tile[R * PITCH];

  const int64_t w0 = w_first + (int64_t)blockIdx.x * WB;
  const int cb0 = blockIdx.y * CB;
  const int64_t rbytes = F32 ? (int64_t)nchans * 4 : ((int64_t)nchans * NBITS + 7) / 8;
  const int64_t b0 = F32 ? (int64_t)cb0 * 4 : (int64_t)cb0 * NBITS / 8;
  // raw row of image sample s: t_begin + s - kPad
  const int64_t r0 = t_begin + w0 * SPW - kPad;

  for (int e = threadIdx.x; e < R * ROWB; e += 256) {
    const int rr = e / ROWB;
    const int bb = e - rr * ROWB;
    const int64_t r = r0 + rr;
    const int64_t byte = b0 + bb;
    uint8_t v = 0;
    if (r >= t_begin && r < t_begin + nrows_valid && byte < rbytes) v = in[r * in_stride + byte];
    tile[rr * PITCH + bb] = v;
  }
  __syncthreads();

  for (int e = threadIdx.x; e < CB * WB; e += 256) {
    const int cl = e / WB;
    const int wl = e - cl * WB;
    const int c = cb0 + cl;
    const int64_t w = w0 + wl;
    if (c >= nchans || w >= words) continue;
    uint32_t word = 0;
    if (F32) {
      const int rr = wl;
      word = *reinterpret_cast<const uint32_t*>(&tile[rr * PITCH + cl * 4]);
    } else {
      const int bitpos = cl * NBITS;
#pragma unroll
      for (int i = 0; i < SPW; ++i) {
        const int rr = wl * SPW + i;
        const uint32_t byte = tile[rr * PITCH + (bitpos >> 3)];
        const uint32_t v = (byte >> (bitpos & 7)) & ((1u << NBITS) - 1u);
        word |= v << (i * LW);
      }
    }
    if (mask && mask[c] == 0) word = 0;
    img[(int64_t)c * row_words + w] = word;
  }
}

// 2-bit input, 1024-byte-aligned rows: the common survey case, specialised.
// Block = 256 threads over 128 channels (32 input bytes per row) x 256 rows
// (32 image words).  Phase 1: each thread loads one row's 32 bytes with two
// 16-byte loads and stores them transposed (byte column major), so the 8
// rows of one image word of a byte column are 8 consecutive bytes.  Phase 2:
// a warp owns one byte column (4 channels) x 32 image words; a lane reads its
// 8 bytes with one 64-bit load and spreads each channel's 2-bit fields to
// 4-bit lanes: (x >> 2k) & 0x03.. keeps channel k in every byte, folding the
// odd bytes into the even bytes' high nibbles and keeping bytes 0, 2, 4, 6
// gives the word.  Requires in, in_stride 16-byte aligned, nchans % 128 == 0.
__global__ void __launch_bounds__(256) k_corner_turn_2bit(const uint8_t* __restrict__ in,
                                                          int64_t in_stride, int64_t t_begin,
                                                          int64_t nrows_valid, int nchans,
                                                          const uint8_t* __restrict__ mask,
                                                          uint32_t* __restrict__ img,
                                                          int64_t row_words, int64_t w_first,
                                                          int64_t words) {
  constexpr int ROWS = 256, COLS = 32, PITCH = ROWS + 8;  // bytes per byte-column row
  __shared__ __align__(16) uint8_t tile[COLS * PITCH];
  const int64_t w0 = w_first + (int64_t)blockIdx.x * 32;  // first image word
  const int cb0 = blockIdx.y * 128;                // first channel
  const int64_t r0 = t_begin + w0 * 8 - kPad;      // raw row of the block's first sample
  {
    const int rr = threadIdx.x;
    const int64_t r = r0 + rr;
    uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
    if (r >= t_begin && r < t_begin + nrows_valid) {
      const uint4* src = reinterpret_cast<const uint4*>(in + r * in_stride + cb0 / 4);
      a = __ldg(src);
      b = __ldg(src + 1);
    }
    const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) tile[(q * 4 + k) * PITCH + rr] = (uint8_t)(v[q] >> (8 * k));
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = w0 + lane;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int col = warp * 4 + it;                 // byte column: channels 4*col .. +3
    const uint2 x = *reinterpret_cast<const uint2*>(&tile[col * PITCH + lane * 8]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = cb0 + col * 4 + k;
      const uint32_t lo = (x.x >> (2 * k)) & 0x03030303u;
      const uint32_t hi = (x.y >> (2 * k)) & 0x03030303u;
      // bytes 0..7 hold the samples; fold byte 2j+1 into byte 2j's high nibble
      const uint32_t flo = lo | (lo >> 4);
      const uint32_t fhi = hi | (hi >> 4);
      uint32_t word = __byte_perm(flo, fhi, 0x6420);
      if (mask && mask[c] == 0) word = 0u;
      if (w < words) img[(int64_t)c * row_words + w] = word;
    }
  }
}

// 8-bit input, 16-byte-aligned rows: the serving bands, specialised.  Block
// = 256 threads over 64 channels (64 input bytes per row) x 64 image words
// (128 rows).  Phase 1: each thread loads 16-byte pieces of rows and stores
// their bytes transposed (channel major), so 8 consecutive samples of one
// channel are 8 consecutive bytes.  Phase 2: a thread reads 8 samples of a
// channel with one 64-bit load and writes the 4 image words they make (two
// 16-bit lanes each) with one 16-byte store.  Requires in, in_stride 16-byte
// aligned, nchans % 64 == 0, row_words and words multiples of 4.
__global__ void __launch_bounds__(256) k_corner_turn_8bit(const uint8_t* __restrict__ in,
                                                          int64_t in_stride, int64_t t_begin,
                                                          int64_t nrows_valid,
                                                          const uint8_t* __restrict__ mask,
                                                          uint32_t* __restrict__ img,
                                                          int64_t row_words, int64_t w_first,
                                                          int64_t words) {
  constexpr int ROWS = 128, CH = 64, PITCH = ROWS + 8;  // bytes per channel row of the tile
  __shared__ __align__(16) uint8_t tile[CH * PITCH];
  const int64_t w0 = w_first + (int64_t)blockIdx.x * 64;  // first image word
  const int cb0 = blockIdx.y * CH;               // first channel
  const int64_t r0 = t_begin + w0 * 2 - kPad;    // raw row of the block's first sample
  for (int e = threadIdx.x; e < ROWS * 4; e += 256) {
    const int rr = e & (ROWS - 1);
    const int pc = e >> 7;  // 16-channel piece of the row
    const int64_t r = r0 + rr;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r >= t_begin && r < t_begin + nrows_valid)
      v = __ldg(reinterpret_cast<const uint4*>(in + r * in_stride + cb0 + 16 * pc));
    const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tile[(16 * pc + 4 * q + k) * PITCH + rr] = (uint8_t)(x[q] >> (8 * k));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < CH * 16; e += 256) {
    const int cl = e >> 4;
    const int qd = e & 15;
    const int64_t w = w0 + 4 * qd;
    if (w >= words) continue;
    const uint2 s = *reinterpret_cast<const uint2*>(&tile[cl * PITCH + 8 * qd]);
    // samples 2i and 2i+1 into the low and high 16-bit lanes of word i
    uint4 o = make_uint4(__byte_perm(s.x, 0u, 0x4140), __byte_perm(s.x, 0u, 0x4342),
                         __byte_perm(s.y, 0u, 0x4140), __byte_perm(s.y, 0u, 0x4342));
    const int c = cb0 + cl;
    if (mask && mask[c] == 0) o = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(img + (int64_t)c * row_words + w) = o;
  }
}

// 8-bit input into 10-bit lanes (three samples a word), 16-byte-aligned
// rows: the serving bands, specialised like the kernel above.  Block = 256
// threads over 64 channels x 64 image words (192 rows).  Phase 1 stores the
// rows' bytes channel major; phase 2: a thread reads 12 samples of a
// channel with three 32-bit loads and writes the 4 image words they make
// with one 16-byte store.  Requires in, in_stride 16-byte aligned, nchans %
// 64 == 0, row_words, w_first and words multiples of 4.
__global__ void __launch_bounds__(256) k_corner_turn_8bit_tri(const uint8_t* __restrict__ in,
                                                              int64_t in_stride, int64_t t_begin,
                                                              int64_t nrows_valid,
                                                              const uint8_t* __restrict__ mask,
                                                              uint32_t* __restrict__ img,
                                                              int64_t row_words, int64_t w_first,
                                                              int64_t words) {
  constexpr int ROWS = 192, CH = 64, PITCH = ROWS + 8;  // bytes per channel row of the tile
  __shared__ __align__(16) uint8_t tile[CH * PITCH];
  const int64_t w0 = w_first + (int64_t)blockIdx.x * 64;  // first image word
  const int cb0 = blockIdx.y * CH;                        // first channel
  const int64_t r0 = t_begin + w0 * 3 - kPad;             // raw row of the block's first sample
  for (int e = threadIdx.x; e < ROWS * 4; e += 256) {
    const int rr = e % ROWS;
    const int pc = e / ROWS;  // 16-channel piece of the row
    const int64_t r = r0 + rr;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r >= t_begin && r < t_begin + nrows_valid)
      v = __ldg(reinterpret_cast<const uint4*>(in + r * in_stride + cb0 + 16 * pc));
    const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tile[(16 * pc + 4 * q + k) * PITCH + rr] = (uint8_t)(x[q] >> (8 * k));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < CH * 16; e += 256) {
    const int cl = e >> 4;
    const int qd = e & 15;
    const int64_t w = w0 + 4 * qd;
    if (w >= words) continue;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&tile[cl * PITCH + 12 * qd]);
    const uint32_t a = src[0], b = src[1], c = src[2];  // samples 0-3, 4-7, 8-11
    // samples 3i, 3i+1, 3i+2 into the 10-bit lanes of word i
    auto s = [&](int k) -> uint32_t {
      const uint32_t x = k < 4 ? a : (k < 8 ? b : c);
      return (x >> (8 * (k & 3))) & 0xFFu;
    };
    uint4 o = make_uint4(s(0) | (s(1) << 10) | (s(2) << 20), s(3) | (s(4) << 10) | (s(5) << 20),
                         s(6) | (s(7) << 10) | (s(8) << 20), s(9) | (s(10) << 10) | (s(11) << 20));
    const int ch = cb0 + cl;
    if (mask && mask[ch] == 0) o = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(img + (int64_t)ch * row_words + w) = o;
  }
}

cudaError_t launch_corner_turn(int nbits, int fmt, const uint8_t* in, int64_t in_stride,
                               int64_t t_begin, int64_t nrows_valid, int nchans,
                               const uint8_t* mask, uint32_t* img, int64_t row_words,
                               int64_t w_first, int64_t words, cudaStream_t st) {
  const int CB = nbits == 32 ? 32 : 256 / nbits;
  const int WB = nbits == 32 ? 64 : 32;
  const bool tri = fmt == FMT_TRI;
  if (tri && nbits != 8) return cudaErrorInvalidValue;
  if (w_first < 0 || w_first >= words) return cudaSuccess;
  const int64_t n = words - w_first;
  dim3 grid((unsigned)((n + WB - 1) / WB), (unsigned)((nchans + CB - 1) / CB));
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  if (grid.y > 65535) return cudaErrorInvalidValue;
  if (nbits == 2 && nchans % 128 == 0 && !(reinterpret_cast<uintptr_t>(in) & 15) &&
      !(in_stride & 15)) {
    const dim3 g2((unsigned)((n + 31) / 32), (unsigned)(nchans / 128));
    k_corner_turn_2bit<<<g2, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, nchans, mask, img,
                                           row_words, w_first, words);
    return cudaGetLastError();
  }
  if (nbits == 8 && nchans % 64 == 0 && !(reinterpret_cast<uintptr_t>(in) & 15) &&
      !(in_stride & 15) && !(row_words & 3) && !(w_first & 3) && !(words & 3) &&
      !(reinterpret_cast<uintptr_t>(img) & 15)) {
    const dim3 g8((unsigned)((n + 63) / 64), (unsigned)(nchans / 64));
    if (tri)
      k_corner_turn_8bit_tri<<<g8, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, mask, img,
                                                 row_words, w_first, words);
    else
      k_corner_turn_8bit<<<g8, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, mask, img,
                                             row_words, w_first, words);
    return cudaGetLastError();
  }
  if (tri) {
    // the generic kernel's block covers 32 image words: 96 rows for 3 samples a word
    k_corner_turn<8, FMT_TRI><<<grid, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, nchans,
                                                    mask, img, row_words, w_first, words);
    return cudaGetLastError();
  }
  switch (nbits) {
    case 1: k_corner_turn<1, FMT_NIB><<<grid, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, nchans, mask, img, row_words, w_first, words); break;
    case 2: k_corner_turn<2, FMT_NIB><<<grid, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, nchans, mask, img, row_words, w_first, words); break;
    case 4: k_corner_turn<4, FMT_BYTE><<<grid, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, nchans, mask, img, row_words, w_first, words); break;
    case 8: k_corner_turn<8, FMT_HALF><<<grid, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, nchans, mask, img, row_words, w_first, words); break;
    case 32: k_corner_turn<32, FMT_F32><<<grid, 256, 0, st>>>(in, in_stride, t_begin, nrows_valid, nchans, mask, img, row_words, w_first, words); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Integer-add probe: each thread runs 8 independent chains of 32-bit adds of
// run-time operands (one PTX add.u32 per counted add).  The result is stored
// so nothing is dead.  Used as the compute roof of the roofline.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_probe_int_add(const uint32_t* __restrict__ seed,
                                                       int64_t iters,
                                                       uint32_t* __restrict__ sink) {
  uint32_t a[8], b[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = seed[k] ^ threadIdx.x;
    b[k] = seed[8 + k] + blockIdx.x;
  }
  for (int64_t it = 0; it < iters; it += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(b[k]));
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= a[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_probe(const uint32_t* seed, int64_t iters, uint32_t* sink, int grid,
                         cudaStream_t st) {
  k_probe_int_add<<<grid, 256, 0, st>>>(seed, iters, sink);
  return cudaGetLastError();
}

}  // namespace dd
