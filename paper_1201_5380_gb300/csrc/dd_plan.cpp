// Plan object: the problem statement of Sec. 2.1 (nu0, dnu, dtau, N_nu and
// the trial list DM(d)), the FP64 delay table of Eq. 3-4, the kill mask and
// the sub-band tables of Sec. 4.1.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "dd_internal.h"

namespace dd {

// k_DM of Eq. 1 (Sec. 1), MHz^2 pc^-1 cm^3 s.
static const double kDispersionConst = 4.148808e3;

DevBuf::~DevBuf() { release(); }
void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}
cudaError_t DevBuf::ensure(size_t n) {
  if (n <= bytes && p) return cudaSuccess;
  release();
  cudaError_t e = cudaMalloc(&p, n ? n : 16);
  if (e != cudaSuccess) {
    p = nullptr;
    return e;
  }
  bytes = n;
  return cudaSuccess;
}

dd_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DD_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return DD_ERR_OOM;
  }
  return DD_ERR_CUDA;
}

int ndm(const Plan& p) { return (int)p.dms.size(); }

static void drain_timing(Plan& p) {
  for (auto& t : p.timed) {
    float ms = 0.f;
    if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      p.timed_ms[t.kind] += ms;
      p.timed_n[t.kind] += 1;
    }
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  p.timed.clear();
  cudaGetLastError();
}

Plan::~Plan() {
  drain_timing(*this);
  for (cudaEvent_t e : part_ev) cudaEventDestroy(e);
  if (copy_st) cudaStreamDestroy(copy_st);
  if (in_st) cudaStreamDestroy(in_st);
}

KernelTimer::KernelTimer(Plan* plan, int k, cudaStream_t s) : p(plan), kind(k), st(s) {
  if (!p || !p->timing) return;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    a = b = nullptr;
    cudaGetLastError();
    return;
  }
  cudaEventRecord(a, st);
}

KernelTimer::~KernelTimer() {
  if (!a) return;
  cudaEventRecord(b, st);
  p->timed.push_back({kind, a, b});
}

// Eq. 3: samples of delay per unit DM for channel c (delay relative to
// channel 0).  The evaluation order (f, then 1/f^2 - 1/f0^2, then the
// k_DM/dtau factor, then the DM product in the caller) is fixed, and the
// library is compiled without FMA contraction, so the table is reproducible.
double partial_delay(double f0, double df, double dt, int c) {
  const double f = f0 + (double)c * df;
  return (kDispersionConst / dt) * (1.0 / (f * f) - 1.0 / (f0 * f0));
}

dd_status build_delays(Plan& p) {
  const int n = ndm(p);
  std::vector<double> dT(p.nchans);
  for (int c = 0; c < p.nchans; ++c) dT[c] = partial_delay(p.f0, p.df, p.dt, c);
  std::vector<int32_t> tab((size_t)n * p.nchans);
  int32_t mx = 0;
  for (int d = 0; d < n; ++d) {
    for (int c = 0; c < p.nchans; ++c) {
      // Eq. 4 with round() read as round-half-up
      const double r = std::floor(p.dms[d] * dT[c] + 0.5);
      if (!(r >= 0.0) || r > 1.0e9) return DD_ERR_INVALID_ARG;
      const int32_t v = (int32_t)r;
      tab[(size_t)d * p.nchans + c] = v;
      if (v > mx) mx = v;
    }
  }
  p.delays.swap(tab);
  p.max_delay = mx;
  for (int i = 0; i < 3; ++i)
    make_blocks(p.delays.data(), n, p.nchans, p.nchans, 16 << i, kSpreadBudget, &p.blocks_B[i],
                &p.spread_B[i], &p.lo_B[i]);
  p.blk_dirty = true;
  p.delays_dirty = true;
  p.sb_dirty = true;
  drop_stage_tabs(p, 7);
  p.scr_dirty = true;
  p.tree_dirty = true;
  return DD_OK;
}

static bool band_ok(int nchans, double dt, double f0, double df) {
  if (nchans <= 0 || nchans > (1 << 20)) return false;
  if (!(dt > 0.0) || !(f0 > 0.0) || !(df < 0.0)) return false;
  if (!(f0 + (double)(nchans - 1) * df > 0.0)) return false;
  return std::isfinite(dt) && std::isfinite(f0) && std::isfinite(df);
}

dd_status ensure_device_tables(Plan& p) {
  if (p.dms.empty()) return DD_ERR_NO_DM_LIST;
  cudaError_t e;
  if (p.delays_dirty || !p.d_delays.p) {
    const size_t nb = p.delays.size() * sizeof(int32_t);
    if ((e = p.d_delays.ensure(nb)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemcpy(p.d_delays.p, p.delays.data(), nb, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cuda_status(e);
    p.delays_dirty = false;
  }
  if (p.mask_dirty || !p.d_mask.p) {
    if ((e = p.d_mask.ensure(p.nchans)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemcpy(p.d_mask.p, p.mask.data(), p.nchans, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cuda_status(e);
    p.mask_dirty = false;
  }
  if (p.blk_dirty) {
    for (int i = 0; i < 3; ++i) {
      const size_t nb = p.blocks_B[i].size() * sizeof(int32_t);
      if ((e = p.d_blk[i].ensure(nb)) != cudaSuccess) return cuda_status(e);
      if ((e = cudaMemcpy(p.d_blk[i].p, p.blocks_B[i].data(), nb, cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return cuda_status(e);
    }
    p.blk_dirty = false;
  }
  if (!p.d_status.p) {
    if ((e = p.d_status.ensure(kStatusBytes)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemset(p.d_status.p, 0, kStatusBytes)) != cudaSuccess)
      return cuda_status(e);
  }
  return DD_OK;
}

// Sub-band tables (Sec. 4.1).  Trials are grouped N'_DM at a time; group g's
// nominal trial is g*N'_DM (its lowest DM, the early-edge alignment of
// App. B) or, centred, the group's middle trial (half the DM error, App. B).
// Stage-1 shifts are differences of rounded delays,
//   rel[g][c] = delay(gn, c) - delay(gn, n0(c)),
// and stage-2 shifts are delay(d, nN'), the telescoped sum of
// Eq. (eq:combining_subbands).
dd_status prepare_subband(Plan& p) {
  if (!p.sb_dirty) return DD_OK;
  if (p.sb_chans <= 0 || p.sb_dms <= 0) return DD_ERR_INVALID_ARG;
  const int n = ndm(p), C = p.nchans, Np = p.sb_chans, nsb = C / Np;
  const int ng = (n + p.sb_dms - 1) / p.sb_dms;
  p.sb_rel.assign((size_t)ng * C, 0);
  p.sb_d2.assign((size_t)n * nsb, 0);
  int32_t mx = 0, m2 = 0;
  for (int g = 0; g < ng; ++g) {
    const int first = g * p.sb_dms, size = std::min(p.sb_dms, n - first);
    const int gn = p.sb_centred ? first + (size - 1) / 2 : first;
    const int32_t* dn = &p.delays[(size_t)gn * C];
    for (int c = 0; c < C; ++c) {
      const int n0 = (c / Np) * Np;
      p.sb_rel[(size_t)g * C + c] = dn[c] - dn[n0];
    }
  }
  for (int d = 0; d < n; ++d) {
    const int g = d / p.sb_dms;
    const int32_t* dd_ = &p.delays[(size_t)d * C];
    for (int s = 0; s < nsb; ++s) {
      const int32_t v = dd_[s * Np];
      p.sb_d2[(size_t)d * nsb + s] = v;
      if (v > m2) m2 = v;
      for (int cp = 0; cp < Np; ++cp) {
        const int32_t r = p.sb_rel[(size_t)g * C + s * Np + cp] + v;
        if (r > mx) mx = r;
      }
    }
  }
  p.sb_max_delay = mx;
  p.sb_len1_extra = m2;
  p.sb_maxrel = 0;
  for (int32_t v : p.sb_rel) p.sb_maxrel = std::max(p.sb_maxrel, v);
  // Trial blocks of each group (sub-band in stage 1, trial group in stage
  // 2), cut to the staging budget; groups with fewer blocks are padded with
  // empty ones so the table is [groups][nblk + 1].
  auto group_tables = [&](int ngrp, int B, auto rows_of, std::vector<int32_t>* table,
                          int32_t* nblk, int32_t* spread, int32_t* lo) {
    std::vector<std::vector<int32_t>> per(ngrp);
    int32_t sp = 0, l = 0, mb = 0;
    for (int g = 0; g < ngrp; ++g) {
      const int32_t* rows;
      int nrows, width, stride;
      rows_of(g, &rows, &nrows, &width, &stride);
      int32_t s1 = 0, l1 = 0;
      make_blocks(rows, nrows, width, stride, B, kSpreadBudget, &per[g], &s1, &l1);
      sp = std::max(sp, s1);
      l = std::max(l, l1);
      mb = std::max(mb, (int32_t)per[g].size() - 1);
    }
    table->assign((size_t)ngrp * (mb + 1), 0);
    for (int g = 0; g < ngrp; ++g) {
      const int nb = (int)per[g].size() - 1;
      for (int b = 0; b <= mb; ++b)
        (*table)[(size_t)g * (mb + 1) + b] = per[g][std::min(b, nb)];
    }
    *nblk = mb;
    *spread = sp;
    *lo = l;
  };
  for (int i = 0; i < 3; ++i) {
    const int B = 16 << i;
    group_tables(
        nsb, B,
        [&](int g, const int32_t** r, int* nr, int* w, int* st) {
          *r = p.sb_rel.data() + (size_t)g * Np;
          *nr = ng;
          *w = Np;
          *st = C;
        },
        &p.sb1_blk_B[i], &p.sb1_nblk_B[i], &p.sb1_spread_B[i], &p.sb1_lo_B[i]);
    group_tables(
        ng, B,
        [&](int g, const int32_t** r, int* nr, int* w, int* st) {
          const int d0 = g * p.sb_dms;
          *r = p.sb_d2.data() + (size_t)d0 * nsb;
          *nr = std::min(p.sb_dms, n - d0);
          *w = nsb;
          *st = nsb;
        },
        &p.sb2_blk_B[i], &p.sb2_nblk_B[i], &p.sb2_spread_B[i], &p.sb2_lo_B[i]);
  }
  p.sb_dirty = false;
  p.sb_dev_dirty = true;
  drop_stage_tabs(p, 6);
  return DD_OK;
}

// Upload the sub-band tables (after prepare_subband).
dd_status upload_subband(Plan& p) {
  dd_status s = prepare_subband(p);
  if (s != DD_OK) return s;
  if (!p.sb_dev_dirty) return DD_OK;
  cudaError_t e;
  if ((e = p.d_sb_rel.ensure(p.sb_rel.size() * 4)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemcpy(p.d_sb_rel.p, p.sb_rel.data(), p.sb_rel.size() * 4,
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_status(e);
  if ((e = p.d_sb_d2.ensure(p.sb_d2.size() * 4)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemcpy(p.d_sb_d2.p, p.sb_d2.data(), p.sb_d2.size() * 4,
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_status(e);
  for (int i = 0; i < 3; ++i) {
    if ((e = p.d_sb1_blk[i].ensure(p.sb1_blk_B[i].size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(p.d_sb1_blk[i].p, p.sb1_blk_B[i].data(), p.sb1_blk_B[i].size() * 4,
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = p.d_sb2_blk[i].ensure(p.sb2_blk_B[i].size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(p.d_sb2_blk[i].p, p.sb2_blk_B[i].data(), p.sb2_blk_B[i].size() * 4,
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_status(e);
  }
  p.sb_dev_dirty = false;
  return DD_OK;
}

bool have_tile_cfg(int B, int K) {
  for (int i = 0; i < kNumTileCfgs; ++i)
    if (kTileCfgs[i].nwarp * kTileCfgs[i].dpw == B && kTileCfgs[i].k == K) return true;
  return false;
}

Tuning tuning_for(const Tuning& t, int fmt) {
  if (t.words_per_lane > 0) return t;
  Tuning r = t;
  // words per lane by accumulator width: 16 where a word's sums take one or
  // two registers (16-bit lanes, 32-bit words), 8 for the 10- and 8-bit
  // lanes' three registers a word (4-bit input on the 1024-channel band to
  // DM 2000, 2^19: 31.6 against 38.3 ms at 4) and for the sub-band stage 2's
  // 8-bit lanes (16 words a lane are compiled for two samples a word at
  // most), 4 for the 4-bit lanes' seven
  const bool one_two = fmt == FMT_HALF || fmt == FMT_U32 || fmt == FMT_F32;
  const bool three = fmt == FMT_TRI || fmt == FMT_BYTE || fmt == FMT_SB8;
  const int prefs[4] = {one_two ? 16 : (three ? 8 : 4), one_two ? 8 : 4, 4, 2};
  for (int k : prefs)
    if (have_tile_cfg(t.dms_per_block, k)) {
      r.words_per_lane = k;
      return r;
    }
  r.words_per_lane = kTileCfgs[0].k;
  r.dms_per_block = kTileCfgs[0].nwarp * kTileCfgs[0].dpw;
  return r;
}

void plan_init_band(Plan& p, int nchans, double dt, double f0, double df) {
  p.nchans = nchans;
  p.dt = dt;
  p.f0 = f0;
  p.df = df;
  p.mask.assign(nchans, 1);
  if (cudaGetDevice(&p.device) != cudaSuccess) p.device = 0;
  cudaGetLastError();
  if (cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device) !=
      cudaSuccess)
    p.num_sms = 0;
  cudaGetLastError();
}

int tile_cfg_index(const Tuning& t0) {
  const Tuning t = t0.words_per_lane > 0 ? t0 : tuning_for(t0, FMT_NIB);
  for (int i = 0; i < kNumTileCfgs; ++i) {
    const TileCfg& c = kTileCfgs[i];
    if (c.nwarp * c.dpw == t.dms_per_block && c.k == t.words_per_lane) return i;
  }
  return 0;
}

}  // namespace dd

using namespace dd;

extern "C" {

const char* dd_status_string(dd_status s) {
  switch (s) {
    case DD_OK: return "ok";
    case DD_ERR_INVALID_ARG: return "invalid argument";
    case DD_ERR_NO_DM_LIST: return "no DM list set";
    case DD_ERR_UNSUPPORTED_NBITS: return "unsupported bits per sample";
    case DD_ERR_INPUT_TOO_SHORT: return "input shorter than nsamps_out + max_delay";
    case DD_ERR_OOM: return "out of memory";
    case DD_ERR_CUDA: return "CUDA error";
    case DD_ERR_TIMEOUT: return "timed out";
    case DD_ERR_DEVICE_BOUNDS: return "device-side bound violation";
    case DD_ERR_OVERFLOW: return "sum could overflow 32 bits";
    case DD_ERR_NOT_READY: return "not ready";
    case DD_ERR_REJECTED: return "rejected by admission control";
  }
  return "unknown status";
}

dd_status dd_plan_create(dd_plan* out, int nchans, double dt_s, double f0_mhz, double df_mhz) {
  if (!out) return DD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!band_ok(nchans, dt_s, f0_mhz, df_mhz)) return DD_ERR_INVALID_ARG;
  Plan* p = new (std::nothrow) Plan();
  if (!p) return DD_ERR_OOM;
  plan_init_band(*p, nchans, dt_s, f0_mhz, df_mhz);
  *out = reinterpret_cast<dd_plan>(p);
  return DD_OK;
}

void dd_plan_destroy(dd_plan plan) { delete reinterpret_cast<Plan*>(plan); }

dd_status dd_plan_set_dm_list(dd_plan plan, const double* dms, int n) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !dms || n <= 0) return DD_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(dms[i]) || dms[i] < 0.0) return DD_ERR_INVALID_ARG;
    if (i && dms[i] < dms[i - 1]) return DD_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(p->mu);
  std::vector<double> old;
  old.swap(p->dms);
  p->dms.assign(dms, dms + n);
  dd_status s = build_delays(*p);
  if (s != DD_OK) {
    p->dms.swap(old);
    build_delays(*p);
  }
  return s;
}

// Trial-DM rule (reading of Sec. 5.2): the next trial is the larger root of
// t_s^2 + w^2 + a^2 x^2 + b^2 (x - DM_i)^2 = tol^2 (t_s^2 + w^2 + a^2 DM_i^2),
// a = 2 k_DM |dnu| / nu_c^3 (us per unit DM, nu_c in GHz), b = a N_nu / 4.
dd_status dd_plan_generate_dm_list(dd_plan plan, double dm_lo, double dm_hi, double width_us,
                                   double tol) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !(dm_lo >= 0.0) || !(dm_hi > dm_lo) || !(tol > 1.0) || !(width_us >= 0.0))
    return DD_ERR_INVALID_ARG;
  const double nu_c = (p->f0 + 0.5 * (double)(p->nchans - 1) * p->df) / 1000.0;
  const double a = 2.0 * kDispersionConst * std::fabs(p->df) / (nu_c * nu_c * nu_c) * 1.0e-3;
  const double b = a * (double)p->nchans / 4.0;
  const double ts = p->dt * 1.0e6;
  const double base = ts * ts + width_us * width_us;
  std::vector<double> out;
  double dm = dm_lo;
  while (dm < dm_hi) {
    out.push_back(dm);
    if (out.size() > 10000000) return DD_ERR_INVALID_ARG;
    const double qa = a * a + b * b;
    const double qb = -2.0 * b * b * dm;
    const double qc = b * b * dm * dm + base - tol * tol * (base + a * a * dm * dm);
    const double disc = qb * qb - 4.0 * qa * qc;
    if (!(disc >= 0.0)) return DD_ERR_INVALID_ARG;
    const double next = (-qb + std::sqrt(disc)) / (2.0 * qa);
    if (!(next > dm)) return DD_ERR_INVALID_ARG;
    dm = next;
  }
  return dd_plan_set_dm_list(plan, out.data(), (int)out.size());
}

dd_status dd_plan_set_killmask(dd_plan plan, const uint8_t* mask) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(p->mu);
  for (int c = 0; c < p->nchans; ++c) p->mask[c] = mask ? (mask[c] ? 1 : 0) : 1;
  p->mask_dirty = true;
  p->scr_dirty = true;
  return DD_OK;
}

dd_status dd_plan_set_gulp(dd_plan plan, int64_t gulp) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || gulp <= 0) return DD_ERR_INVALID_ARG;
  p->gulp = gulp;
  return DD_OK;
}

dd_status dd_plan_set_subband_alignment(dd_plan plan, int centred) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || (centred != 0 && centred != 1)) return DD_ERR_INVALID_ARG;
  if (p->sb_centred != (centred == 1)) {
    p->sb_centred = centred == 1;
    p->sb_dirty = true;
  }
  return DD_OK;
}

dd_status dd_plan_set_subband(dd_plan plan, int chans_per_sb, int dms_per_nom) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DD_ERR_INVALID_ARG;
  if (chans_per_sb == 0 && dms_per_nom == 0) {
    p->sb_chans = p->sb_dms = 0;
    return DD_OK;
  }
  if (chans_per_sb <= 0 || dms_per_nom <= 0 || p->nchans % chans_per_sb != 0)
    return DD_ERR_INVALID_ARG;
  p->sb_chans = chans_per_sb;
  p->sb_dms = dms_per_nom;
  p->sb_dirty = true;
  return DD_OK;
}

dd_status dd_plan_set_tuning(dd_plan plan, int dms_per_block, int cc, int words) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DD_ERR_INVALID_ARG;
  Tuning t = p->tune;
  if (dms_per_block) t.dms_per_block = dms_per_block;
  if (cc) t.chans_per_chunk = cc;
  if (words > 0) t.words_per_lane = words;
  if (words < 0) t.words_per_lane = 0;  // per input format
  if (t.chans_per_chunk < 4 || t.chans_per_chunk > 32 ||
      (t.chans_per_chunk & (t.chans_per_chunk - 1)))
    return DD_ERR_INVALID_ARG;
  bool found = false;
  for (int i = 0; i < kNumTileCfgs; ++i)
    if (kTileCfgs[i].nwarp * kTileCfgs[i].dpw == t.dms_per_block &&
        (t.words_per_lane == 0 || kTileCfgs[i].k == t.words_per_lane))
      found = true;
  if (!found) return DD_ERR_INVALID_ARG;
  p->tune = t;
  p->scr_dirty = true;
  return DD_OK;
}

dd_status dd_plan_get_tuning(dd_plan plan, int* dms_per_block, int* cc, int* words) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DD_ERR_INVALID_ARG;
  if (dms_per_block) *dms_per_block = p->tune.dms_per_block;
  if (cc) *cc = p->tune.chans_per_chunk;
  if (words) *words = p->tune.words_per_lane;
  return DD_OK;
}

dd_status dd_plan_get_dm_count(dd_plan plan, int32_t* n) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !n) return DD_ERR_INVALID_ARG;
  *n = (int32_t)p->dms.size();
  return DD_OK;
}

dd_status dd_plan_get_dm_list(dd_plan plan, double* out) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !out) return DD_ERR_INVALID_ARG;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  std::memcpy(out, p->dms.data(), p->dms.size() * sizeof(double));
  return DD_OK;
}

dd_status dd_plan_get_max_delay(dd_plan plan, int32_t* m) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !m) return DD_ERR_INVALID_ARG;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  *m = p->max_delay;
  return DD_OK;
}

dd_status dd_plan_get_subband_max_delay(dd_plan plan, int32_t* m) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !m) return DD_ERR_INVALID_ARG;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  if (p->sb_chans <= 0) return DD_ERR_INVALID_ARG;
  if (p->sb_dirty) {
    dd_status s = prepare_subband(*p);
    if (s != DD_OK) return s;
  }
  *m = p->sb_max_delay;
  return DD_OK;
}

dd_status dd_plan_get_delay_table(dd_plan plan, int32_t* out) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !out) return DD_ERR_INVALID_ARG;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  std::memcpy(out, p->delays.data(), p->delays.size() * sizeof(int32_t));
  return DD_OK;
}

dd_status dd_plan_set_kernel_timing(dd_plan plan, int enable) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DD_ERR_INVALID_ARG;
  p->timing = enable != 0;
  return DD_OK;
}

dd_status dd_plan_get_kernel_timing(dd_plan plan, int kind, double* total_ms, int64_t* launches) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || kind < 0 || kind > 2) return DD_ERR_INVALID_ARG;
  drain_timing(*p);
  if (total_ms) *total_ms = p->timed_ms[kind];
  if (launches) *launches = p->timed_n[kind];
  return DD_OK;
}

dd_status dd_plan_reset_kernel_timing(dd_plan plan) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DD_ERR_INVALID_ARG;
  drain_timing(*p);
  for (int k = 0; k < 3; ++k) {
    p->timed_ms[k] = 0.0;
    p->timed_n[k] = 0;
  }
  return DD_OK;
}

dd_status dd_plan_get_device_status(dd_plan plan, uint32_t* flags) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !flags) return DD_ERR_INVALID_ARG;
  *flags = 0;
  if (!p->d_status.p) return DD_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t v = 0;
  if ((e = cudaMemcpy(&v, p->d_status.p, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMemset(p->d_status.p, 0, 4)) != cudaSuccess) return cuda_status(e);
  *flags = v;
  return DD_OK;
}

}  // extern "C"
