// Time-scrunching (Sec. 2.2): beyond twice the diagonal DM a trial is
// dedispersed at half the time resolution, and again at each further
// doubling: the input is summed over s adjacent samples and Eq. 3-4 is
// evaluated at s*dt.  Trials of one factor s form a level, run by a child
// plan of resolution s*dt over the level's trials; row d of the output then
// holds nsamps_out / s_d samples.
//
// The diagonal DM is where the delays of the top two channels (the smallest
// per-channel step) differ by one sample: 1 / ((k_DM/dt) (1/f1^2 - 1/f0^2)).
// Scrunched samples of 1/2/4-bit input fit 4 bits while s * max <= 15 (the
// child then reads 4-bit packed input, 8-bit lanes) and 8 bits up to s = 16.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "dd_internal.h"

namespace dd {
namespace {

constexpr double kScrunchDispersion = 4.148808e3;  // k_DM, MHz^2 pc^-1 cm^3 s (Sec. 1)

// One thread per output byte: NB_OUT = 8 holds one channel, 4 holds two.
template <int NB_IN, int NB_OUT>
__global__ void __launch_bounds__(256) k_scrunch(const uint8_t* __restrict__ in, int64_t in_stride,
                                                 int s, int64_t rows_out, int nchans,
                                                 uint8_t* __restrict__ out, int64_t out_stride,
                                                 int64_t out_row_bytes) {
  const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (idx >= rows_out * out_row_bytes) return;
  const int64_t r = idx / out_row_bytes;
  const int b = (int)(idx - r * out_row_bytes);
  constexpr int PER = 8 / NB_OUT;  // channels per output byte
  uint32_t byte = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int c = b * PER + k;
    if (c >= nchans) break;
    const int64_t cb = (int64_t)c * NB_IN / 8;
    const int sh = (c * NB_IN) & 7;
    uint32_t sum = 0;
    for (int u = 0; u < s; ++u)
      sum += ((uint32_t)in[((int64_t)s * r + u) * in_stride + cb] >> sh) & ((1u << NB_IN) - 1u);
    byte |= sum << (k * NB_OUT);
  }
  out[r * out_stride + b] = (uint8_t)byte;
}

cudaError_t launch_scrunch(int nb_in, int nb_out, int s, const uint8_t* in, int64_t in_stride,
                           int64_t rows_out, int nchans, uint8_t* out, int64_t out_row_bytes,
                           cudaStream_t st) {
  const int64_t total = rows_out * out_row_bytes;
  if (total == 0) return cudaSuccess;
  const dim3 grid((unsigned)((total + 255) / 256));
#define DD_SCR(NI, NO)                                                                     \
  if (nb_in == NI && nb_out == NO) {                                                       \
    k_scrunch<NI, NO><<<grid, 256, 0, st>>>(in, in_stride, s, rows_out, nchans, out,       \
                                           out_row_bytes, out_row_bytes);                  \
    return cudaGetLastError();                                                             \
  }
  DD_SCR(1, 4)
  DD_SCR(1, 8)
  DD_SCR(2, 4)
  DD_SCR(2, 8)
  DD_SCR(4, 8)
#undef DD_SCR
  return cudaErrorInvalidValue;
}

int out_bits(int nbits, int s) { return s * vmax_for_nbits(nbits) <= 15 ? 4 : 8; }

}  // namespace

dd_status prepare_scrunch(Plan& p) {
  if (!p.scr_dirty) return DD_OK;
  if (p.scrunch_max < 1 || p.dms.empty()) return DD_ERR_INVALID_ARG;
  const double f0 = p.f0, f1 = p.f0 + 1.0 * p.df;
  const double step = (kScrunchDispersion / p.dt) * (1.0 / (f1 * f1) - 1.0 / (f0 * f0));
  const double diag = step > 0.0 ? 1.0 / step : 0.0;
  const int n = (int)p.dms.size();
  p.scr_factor.assign(n, 1);
  for (int d = 0; d < n; ++d) {
    int s = 1;
    while (s < p.scrunch_max && diag > 0.0 && p.dms[d] >= 2.0 * (double)s * diag) s *= 2;
    p.scr_factor[d] = s;
  }
  p.scr_levels.clear();
  int d0 = 0;
  while (d0 < n) {
    int d1 = d0 + 1;
    while (d1 < n && p.scr_factor[d1] == p.scr_factor[d0]) ++d1;
    Plan::ScrLevel L;
    L.s = p.scr_factor[d0];
    L.d_lo = d0;
    L.d_hi = d1;
    L.plan.reset(new Plan());
    Plan& c = *L.plan;
    plan_init_band(c, p.nchans, p.dt * L.s, p.f0, p.df);
    c.mask = p.mask;
    c.tune = p.tune;
    c.dms.assign(p.dms.begin() + d0, p.dms.begin() + d1);
    dd_status st = build_delays(c);
    if (st != DD_OK) {
      p.scr_levels.clear();
      return st;
    }
    p.scr_levels.push_back(std::move(L));
    d0 = d1;
  }
  p.scr_dirty = false;
  return DD_OK;
}

// Input rows the scrunched transform reads: level s needs s rows for each of
// its nsamps_out / s + max_delay scrunched samples.
int64_t scrunch_input_rows(const Plan& p, int64_t nsamps_out) {
  int64_t rows = 0;
  for (const Plan::ScrLevel& L : p.scr_levels) {
    const int64_t n = nsamps_out / L.s;
    if (n == 0) continue;
    rows = std::max<int64_t>(rows, (int64_t)L.s * (n + L.plan->max_delay));
  }
  return rows;
}

dd_status exec_scrunch(Plan& p, const ExecArgs& a) {
  if (a.in_nbits > 4) return DD_ERR_UNSUPPORTED_NBITS;
  dd_status s = prepare_scrunch(p);
  if (s != DD_OK) return s;
  if (a.in_rows < scrunch_input_rows(p, a.nsamps_out)) return DD_ERR_INPUT_TOO_SHORT;
  for (Plan::ScrLevel& L : p.scr_levels) {
    Plan& c = *L.plan;
    const int64_t n = a.nsamps_out / L.s;
    if (n == 0) continue;
    ExecArgs b = a;
    b.nsamps_out = n;
    b.out = static_cast<uint32_t*>(a.out) + (int64_t)L.d_lo * a.out_stride;
    b.subband = false;
    if (L.s > 1) {
      const int nb = out_bits(a.in_nbits, L.s);
      const int64_t rows = n + c.max_delay;
      const int64_t rb = ((int64_t)p.nchans * nb + 7) / 8;
      cudaError_t e = p.d_scr.ensure((size_t)(rows * rb));
      if (e != cudaSuccess) return cuda_status(e);
      e = launch_scrunch(a.in_nbits, nb, L.s, static_cast<const uint8_t*>(a.in),
                         a.in_row_stride, rows, p.nchans, static_cast<uint8_t*>(p.d_scr.p), rb,
                         a.st);
      if (e != cudaSuccess) return cuda_status(e);
      b.in = p.d_scr.p;
      b.in_nbits = nb;
      b.in_row_stride = rb;
      b.in_rows = rows;
    }
    if ((s = exec_device(c, b)) != DD_OK) return s;
  }
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_plan_set_scrunch(dd_plan plan, int max_factor) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DD_ERR_INVALID_ARG;
  if (max_factor != 0 && (max_factor < 1 || max_factor > 16 || (max_factor & (max_factor - 1))))
    return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(p->mu);
  p->scrunch_max = max_factor;
  p->scr_dirty = true;
  return DD_OK;
}

dd_status dd_plan_get_scrunch_factors(dd_plan plan, int32_t* factors) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !factors) return DD_ERR_INVALID_ARG;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  std::lock_guard<std::mutex> lk(p->mu);
  if (p->scrunch_max == 0) {
    std::fill(factors, factors + p->dms.size(), 1);
    return DD_OK;
  }
  dd_status s = prepare_scrunch(*p);
  if (s != DD_OK) return s;
  std::copy(p->scr_factor.begin(), p->scr_factor.end(), factors);
  return DD_OK;
}

}  // extern "C"
