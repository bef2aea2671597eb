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
// sums (N' * max sample) stay below 2^16.
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
__host__ __device__ constexpr int tree_words(int nsub) { return ((tree_tile(nsub) + nsub) / 2) | 1; }  // odd pitch
constexpr int kTreeThreads = 256;
constexpr int kMaxTreeChans = 128;

struct TreeS1 {
  const uint8_t* in;      // packed time-major rows
  int64_t in_stride;      // bytes per row
  int64_t in_rows;        // valid rows (zeros beyond)
  const uint8_t* mask;    // nchans, 0 = killed
  uint32_t* S;            // stage-1 rows, two 16-bit samples per word
  int64_t s_pitch;        // words per S row
  const int32_t* roff;    // first S row of each sub-band (+ end)
  int64_t len1;           // samples per S row that stage 2 reads
  int nbits;
};

// Eq. (shuffle) and Eq. (tree_integer_delay), truncated divisions.
__device__ __forceinline__ int tree_phi(int r, int v) { return (v & 1) * r + v / 2 + (v / (2 * r)) * r; }
__device__ __forceinline__ int tree_theta(int r, int v) { return ((v & (2 * r - 1)) + 1) >> 1; }

template <int NSUB>
__global__ void __launch_bounds__(kTreeThreads) k_tree_stage1(const TreeS1 p) {
  constexpr int T = tree_tile(NSUB);
  constexpr int WW = tree_words(NSUB);
  extern __shared__ uint32_t sm[];
  uint32_t* buf0 = sm;
  uint32_t* buf1 = sm + NSUB * WW;
  const int n = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * T;
  const int tid = threadIdx.x;
  const int c0 = n * NSUB;
  const uint32_t vmask = (1u << p.nbits) - 1u;

  // (a) unpack rows t0 .. t0 + 2 WW - 1 of the sub-band's channels into 16-bit
  //     lanes (consecutive threads take consecutive channels of one row)
  {
    uint16_t* a16 = reinterpret_cast<uint16_t*>(buf0);
    for (int e = tid; e < NSUB * 2 * WW; e += kTreeThreads) {
      const int c = e % NSUB;
      const int tl = e / NSUB;
      const int64_t t = t0 + tl;
      uint32_t v = 0u;
      if (t < p.in_rows) {
        const int64_t bit = (int64_t)(c0 + c) * p.nbits;
        const uint8_t byte = __ldg(p.in + t * p.in_stride + (bit >> 3));
        v = ((uint32_t)byte >> (bit & 7)) & vmask;
        if (!__ldg(p.mask + c0 + c)) v = 0u;
      }
      a16[c * 2 * WW + tl] = (uint16_t)v;
    }
  }
  __syncthreads();

  // (b) the log2 N' steps, out of place between the two buffers
  uint32_t* src = buf0;
  uint32_t* dst = buf1;
#pragma unroll 1
  for (int r = 1; r < NSUB; r *= 2) {
    for (int e = tid; e < NSUB * WW; e += kTreeThreads) {
      const int o = e / WW;
      const int q = e - o * WW;
      const int v = o >> 1;
      const uint32_t* lo = src + tree_phi(r, 2 * v) * WW;
      const uint32_t* hi = src + tree_phi(r, 2 * v + 1) * WW;
      const int th = tree_theta(r, o);
      const int qq = q + (th >> 1);
      // words past the buffer hold samples beyond the loaded rows: every
      // output they reach is past the tile's last sample (t0 + T - 1 needs
      // input only up to t0 + T + N' - 2 < t0 + 2 WW)
      const uint32_t b0 = qq < WW ? hi[qq] : 0u;
      uint32_t b = b0;
      if (th & 1) {
        const uint32_t b1 = qq + 1 < WW ? hi[qq + 1] : 0u;
        b = __funnelshift_r(b0, b1, 16);
      }
      dst[o * WW + q] = lo[q] + b;
    }
    __syncthreads();
    uint32_t* sw = src;
    src = dst;
    dst = sw;
  }

  // (c) the trails stage 2 reads, T samples of each
  const int r0 = __ldg(p.roff + n);
  const int nrow = __ldg(p.roff + n + 1) - r0;
  const int64_t w0 = t0 / 2;
  const int64_t wend = (p.len1 + 1) / 2;
  for (int e = tid; e < nrow * (T / 2); e += kTreeThreads) {
    const int d = e / (T / 2);
    const int q = e - d * (T / 2);
    if (w0 + q < wend) p.S[(int64_t)(r0 + d) * p.s_pitch + w0 + q] = src[d * WW + q];
  }
}

struct TreeS2 {
  const uint16_t* S;      // stage-1 rows, 16-bit samples
  int64_t s_pitch;        // samples per S row
  const int2* tab;        // [trial][sub-band] {S row, shift}
  int nsb, ndm;
  int64_t nsamps;
  uint32_t* out;
  int64_t out_stride;
};

constexpr int kS2Warps = 8;  // trials per block
constexpr int kS2K = 8;      // samples per lane (stride 32)

__global__ void __launch_bounds__(kS2Warps * 32) k_tree_stage2(const TreeS2 p) {
  extern __shared__ int2 s_tab[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int d0 = blockIdx.y * kS2Warps;
  const int64_t t0 = (int64_t)blockIdx.x * (32 * kS2K);
  const int nd = min(kS2Warps, p.ndm - d0);
  for (int e = threadIdx.x; e < nd * p.nsb; e += blockDim.x)
    s_tab[e] = p.tab[(int64_t)d0 * p.nsb + e];
  __syncthreads();
  if (warp >= nd) return;
  const int d = d0 + warp;
  uint32_t acc[kS2K];
#pragma unroll
  for (int j = 0; j < kS2K; ++j) acc[j] = 0u;
  const int2* tab = s_tab + warp * p.nsb;
  // samples past the gulp are neither read nor written (their reads could
  // pass the end of the last stage-1 row)
  const int64_t left = p.nsamps - t0 - lane;
  for (int n = 0; n < p.nsb; ++n) {
    const int2 rs = tab[n];
    const uint16_t* row = p.S + (int64_t)rs.x * p.s_pitch + rs.y + t0 + lane;
#pragma unroll
    for (int j = 0; j < kS2K; ++j)
      if (32 * j < left) acc[j] += __ldg(row + 32 * j);
  }
  uint32_t* o = p.out + (int64_t)d * p.out_stride + t0 + lane;
#pragma unroll
  for (int j = 0; j < kS2K; ++j)
    if (t0 + lane + 32 * j < p.nsamps) o[32 * j] = acc[j];
}

template <int NSUB>
cudaError_t launch_stage1(const TreeS1& a, int64_t tiles, int nsb, cudaStream_t st) {
  const size_t smem = 2u * NSUB * tree_words(NSUB) * 4u;
  auto k = k_tree_stage1<NSUB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<dim3((unsigned)tiles, (unsigned)nsb), kTreeThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t stage1(int nsub, const TreeS1& a, int64_t tiles, int nsb, cudaStream_t st) {
  switch (nsub) {
    case 2: return launch_stage1<2>(a, tiles, nsb, st);
    case 4: return launch_stage1<4>(a, tiles, nsb, st);
    case 8: return launch_stage1<8>(a, tiles, nsb, st);
    case 16: return launch_stage1<16>(a, tiles, nsb, st);
    case 32: return launch_stage1<32>(a, tiles, nsb, st);
    case 64: return launch_stage1<64>(a, tiles, nsb, st);
    case 128: return launch_stage1<128>(a, tiles, nsb, st);
    default: return cudaErrorInvalidValue;
  }
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
  if ((e = p.d_tree_S.ensure((size_t)rows * pitch * 2)) != cudaSuccess) return cuda_status(e);
  TreeS1 s1;
  s1.in = static_cast<const uint8_t*>(a.in);
  s1.in_stride = a.in_row_stride;
  s1.in_rows = a.in_rows;
  s1.mask = static_cast<const uint8_t*>(p.d_mask.p);
  s1.S = static_cast<uint32_t*>(p.d_tree_S.p);
  s1.s_pitch = pitch / 2;
  s1.roff = static_cast<const int32_t*>(p.d_tree_roff.p);
  s1.len1 = len1;
  s1.nbits = a.in_nbits;
  {
    KernelTimer kt(&p, DD_KERNEL_DEDISP, a.st);
    if ((e = stage1(Np, s1, tiles, nsb, a.st)) != cudaSuccess) return cuda_status(e);
  }
  TreeS2 s2;
  s2.S = static_cast<const uint16_t*>(p.d_tree_S.p);
  s2.s_pitch = pitch;
  s2.tab = static_cast<const int2*>(p.d_tree_tab.p);
  s2.nsb = nsb;
  s2.ndm = n;
  s2.nsamps = a.nsamps_out;
  s2.out = static_cast<uint32_t*>(a.out);
  s2.out_stride = a.out_stride;
  const int64_t t2 = (a.nsamps_out + 32 * kS2K - 1) / (32 * kS2K);
  const dim3 grid((unsigned)t2, (unsigned)((n + kS2Warps - 1) / kS2Warps));
  const size_t smem = (size_t)kS2Warps * nsb * sizeof(int2);
  KernelTimer kt(&p, DD_KERNEL_STAGE2, a.st);
  k_tree_stage2<<<grid, kS2Warps * 32, smem, a.st>>>(s2);
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
