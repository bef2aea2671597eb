// Execution: corner turn into the staged image, then the direct kernel over
// a list of work segments (direct: one segment; sub-band: one segment per
// sub-band for stage 1 and one per trial group for stage 2, Sec. 4.1).
#include <dlfcn.h>

#include <algorithm>
#include <climits>
#include <cstring>

#include "dd_internal.h"

namespace dd {

int fmt_for_nbits(int nbits, int nchans) {
  switch (nbits) {
    case 1:
    case 2: return FMT_NIB;
    case 4: return FMT_BYTE;
    case 8: return (int64_t)nchans * 255 < ((int64_t)1 << 20) ? FMT_TRI : FMT_HALF;
    case 32: return FMT_F32;
    default: return -1;
  }
}

int vmax_for_nbits(int nbits) { return nbits == 32 ? 0 : (1 << nbits) - 1; }

// Largest staging spread of any (trial block, channel): max_d delay(d,c) -
// delay(d0,c) + lo_slack, where lo_slack covers trials whose delay is below
// the block's first (sub-band stage-1 tables are only nearly monotone).
int32_t max_block_spread(const int32_t* delays, int ndm, int nchans, int stride, int B,
                         int32_t* lo_slack) {
  int32_t spread = 0, lo = 0;
  for (int d0 = 0; d0 < ndm; d0 += B) {
    const int d1 = std::min(ndm, d0 + B);
    for (int c = 0; c < nchans; ++c) {
      const int32_t s0 = delays[(size_t)d0 * stride + c];
      int32_t mn = s0, mx = s0;
      for (int d = d0 + 1; d < d1; ++d) {
        const int32_t s = delays[(size_t)d * stride + c];
        mn = std::min(mn, s);
        mx = std::max(mx, s);
      }
      lo = std::max(lo, s0 - mn);
      spread = std::max(spread, mx - s0);
    }
  }
  *lo_slack = lo;
  return spread + lo;
}

void make_blocks(const int32_t* delays, int ndm, int nchans, int stride, int B, int32_t budget,
                 std::vector<int32_t>* starts, int32_t* spread_out, int32_t* lo_out) {
  starts->clear();
  int32_t spread_all = 0, lo_all = 0;
  std::vector<int32_t> mn(nchans), mx(nchans);
  int d0 = 0;
  while (d0 < ndm) {
    starts->push_back(d0);
    const int32_t* r0 = delays + (size_t)d0 * stride;
    for (int c = 0; c < nchans; ++c) mn[c] = mx[c] = r0[c];
    int32_t sp = 0, lo = 0;
    int d = d0 + 1;
    for (; d < ndm && d < d0 + B; ++d) {
      const int32_t* r = delays + (size_t)d * stride;
      int32_t sp2 = 0, lo2 = 0;
      for (int c = 0; c < nchans; ++c) {
        const int32_t a = std::min(mn[c], r[c]), b = std::max(mx[c], r[c]);
        lo2 = std::max(lo2, r0[c] - a);
        sp2 = std::max(sp2, b - r0[c]);
      }
      if (sp2 + lo2 > budget) break;
      for (int c = 0; c < nchans; ++c) {
        mn[c] = std::min(mn[c], r[c]);
        mx[c] = std::max(mx[c], r[c]);
      }
      sp = sp2;
      lo = lo2;
    }
    spread_all = std::max(spread_all, sp + lo);
    lo_all = std::max(lo_all, lo);
    d0 = d;
  }
  starts->push_back(ndm);
  *spread_out = spread_all;
  *lo_out = lo_all;
}

int time_tile(int fmt, const Tuning& t) { return 32 * t.words_per_lane * fmt_spw(fmt); }

static int window_words(int fmt, const Tuning& t, int32_t spread) {
  const int spw = fmt_spw(fmt);
  int nww = (4 * spw - 1 + spread) / spw + 32 * t.words_per_lane;
  return (nww + 3) & ~3;
}

// Image row pitch (words) covering every staging read of a job with nsamps
// outputs, largest delay maxd and staging spread `spread`.
int64_t image_row_words(int fmt, const Tuning& t, int64_t nsamps, int32_t maxd,
                        int32_t spread) {
  const int spw = fmt_spw(fmt);
  const int T = time_tile(fmt, t);
  const int64_t tiles = (nsamps + T - 1) / T;
  const int64_t last_sample = tiles * T + kPad + maxd + 4 * spw;
  int64_t w = last_sample / spw + window_words(fmt, t, spread) + 8;
  return (w + 31) & ~(int64_t)31;
}

static void flush_periods(int fmt, int vmax, int nchan_max, bool* wide, int* f0, int* f1,
                          int* f2) {
  *wide = false;
  *f0 = *f1 = *f2 = INT_MAX;
  if (vmax < 1) vmax = 1;
  switch (fmt) {
    case FMT_NIB:
      *f0 = std::max(1, 15 / (4 * vmax));
      *f1 = std::max(1, 255 / (4 * vmax * *f0));
      *f2 = std::max(1, 65535 / (4 * vmax * *f0 * *f1));
      *wide = (int64_t)nchan_max * vmax > 65535;
      break;
    case FMT_BYTE:
      *f0 = std::max(1, 255 / (4 * vmax));
      *f1 = std::max(1, 65535 / (4 * vmax * *f0));
      *wide = (int64_t)nchan_max * vmax > 65535;
      break;
    case FMT_HALF:
      *f0 = std::max(1, 65535 / (4 * vmax));
      *wide = (int64_t)nchan_max * vmax > 65535;
      break;
    case FMT_SB8:
      // pairs of values below 128 spread into 16-bit lanes (no flush)
      *wide = (int64_t)nchan_max * vmax > 65535;
      break;
    case FMT_TRI:
      *f0 = 1;  // every group of 4 channels leaves the 10-bit lanes
      *f1 = 4;  // lane 2 of the separated sums holds four groups
      break;
    case FMT_F32:
      *f0 = 8;  // 32 channels per FP32 partial sum
      break;
    default:
      break;
  }
}

struct SegSpec {
  Seg seg;
  int32_t spread;
  int kind;        // staging-table kind (0 direct, 1/2 sub-band stage)
  Plan* owner;     // plan that caches the staging tables
  TabSrc src;
  bool no_upload;  // tables stay on the host (the caller places them)
  std::shared_ptr<StageTab> tab;  // set by finish_launch
};

// Staging tables (Seg::atab, Seg::crec) of one delay table.  For trial
// block b and channel c the window starts at image word t0/SPW + woff,
// woff = floor((kPad + s0 - lo) / (4 SPW)) * 4 with s0 the block's first
// delay; trial slot i (slots past the block's last trial repeat it) reads
// lane-shifted copy kap = o mod SPW from word o / SPW, o = kPad + s_i -
// woff*SPW.  Each block gets its own chunk geometry: its window width nww
// is the widest read span of its channels, and its chunk the most channels
// (a power of two up to cc_cap; for 4- and 8-bit input a multiple of 4,
// evened out over the chunks it takes) whose two staging buffers fit in shared memory,
// so blocks with a small delay spread stage more channels per barrier than
// the launch's widest block could.  When every block gets the same chunk, all
// of them take the window width nww_uniform instead (at least the widest
// span): one geometry for the launch, which the kernel then reads from its
// parameters rather than per block.  Absent channels of a last partial
// chunk read the zero window.
static dd_status build_stage_tab(const TabSrc& src, int fmt, int cfg, int cc_cap,
                                 int nww_uniform, StageTab* t) {
  const int spw = fmt_spw(fmt);
  const int B = kTileCfgs[cfg].nwarp * kTileCfgs[cfg].dpw;
  const int K = kTileCfgs[cfg].k;
  const int nt = kTileCfgs[cfg].nwarp * 32;
  const bool copies = spw > 1;
  t->g_crec = (int64_t)src.nblk * (src.nchan + 1) * 2;
  t->crec.assign((size_t)(t->g_crec * src.ngroups), 0);
  t->smem = 0;
  t->reach = 0;
  // window start of (block, channel) and the words its trials read
  auto window = [&](const int32_t* dl, int d0, int d1, int c, int64_t* woff,
                    int64_t* span) -> bool {
    const int64_t b0 = (int64_t)kPad + dl[(int64_t)d0 * src.dstride + c] - src.lo;
    if (b0 < 0) return false;
    *woff = b0 / (4 * spw) * 4;
    int64_t sp = 0;
    for (int i = 0; i < B; ++i) {
      const int d = std::min(d0 + i, d1 - 1);
      const int64_t o = (int64_t)kPad + dl[(int64_t)d * src.dstride + c] - *woff * spw;
      if (o < 0) return false;
      sp = std::max<int64_t>(sp, o / spw + 32 * K);
    }
    *span = sp;
    return true;
  };
  auto fits = [&](int cc, int nww) {
    return dedisp_smem_bytes(fmt, cfg, cc, nww) <= kSmemCap && B * cc <= 2 * nt;
  };
  // pass 1: each block's widest span and the chunk it allows
  std::vector<int> bcc((size_t)src.ngroups * src.nblk, 0), bnww(bcc.size(), 0);
  int cc_lo = INT_MAX, cc_hi = 0, nww_hi = 0;
  for (int g = 0; g < src.ngroups; ++g) {
    const int32_t* dl = src.delays + (int64_t)g * src.g_delay;
    const int32_t* bt = src.blk + (int64_t)g * (src.nblk + 1);
    for (int b = 0; b < src.nblk; ++b) {
      const int d0 = bt[b], d1 = bt[b + 1];
      if (d1 <= d0) continue;  // padding block: never visited
      int64_t widest = 0, woff, span;
      for (int c = 0; c < src.nchan; ++c) {
        if (!window(dl, d0, d1, c, &woff, &span)) return DD_ERR_INVALID_ARG;
        widest = std::max(widest, span);
      }
      if (widest > INT_MAX / 64) return DD_ERR_INVALID_ARG;
      const int nww = (int)((widest + 3) & ~3);
      int cc = cc_cap;
      if (fmt == FMT_TRI || fmt == FMT_BYTE) {
        // 4- and 8-bit input (8- and 10-bit lanes): any multiple of 4
        // channels, evened out over the chunks it takes (a smaller last
        // chunk stages fewer absent channels).  On the 1024-channel band to
        // DM 2000 this took 41.4 against 42.5 ms (8-bit) and 31.6 against
        // 32.2 ms (4-bit); the other formats keep powers of two (the survey
        // band: 18.08 against 18.00 ms with multiples of 4).
        while (cc > 4 && !fits(cc, nww)) cc -= 4;
        const int nch = (src.nchan + cc - 1) / cc;
        cc = std::min(cc, ((src.nchan + nch - 1) / nch + 3) & ~3);
      } else {
        while (cc > 4 && !fits(cc, nww)) cc /= 2;
      }
      if (!fits(cc, nww)) return DD_ERR_INVALID_ARG;
      bcc[(size_t)g * src.nblk + b] = cc;
      bnww[(size_t)g * src.nblk + b] = nww;
      cc_lo = std::min(cc_lo, cc);
      cc_hi = std::max(cc_hi, cc);
      nww_hi = std::max(nww_hi, nww);
    }
  }
  t->uniform = cc_hi > 0 && cc_lo == cc_hi;
  if (t->uniform) {
    t->cc = cc_hi;
    t->nww = std::max(nww_hi, (nww_uniform + 3) & ~3);
    if (!fits(t->cc, t->nww)) t->nww = nww_hi;
  }
  // offsets per block: every chunk of the block's chunk size, the last one
  // padded with absent channels
  int64_t per_blk = 0;
  for (size_t i = 0; i < bcc.size(); ++i)
    if (bcc[i] > 0) {
      const int cc = t->uniform ? t->cc : bcc[i];
      per_blk = std::max<int64_t>(per_blk, (int64_t)((src.nchan + cc - 1) / cc) * cc * B);
    }
  t->atab_blk = per_blk;
  t->g_atab = (int64_t)src.nblk * t->atab_blk;
  t->atab.assign((size_t)(t->g_atab * src.ngroups), 0u);
  // pass 2: the tables
  for (int g = 0; g < src.ngroups; ++g) {
    const int32_t* dl = src.delays + (int64_t)g * src.g_delay;
    const int32_t* bt = src.blk + (int64_t)g * (src.nblk + 1);
    for (int b = 0; b < src.nblk; ++b) {
      const int d0 = bt[b], d1 = bt[b + 1];
      if (d1 <= d0) continue;
      const int cc = t->uniform ? t->cc : bcc[(size_t)g * src.nblk + b];
      const int nww = t->uniform ? t->nww : bnww[(size_t)g * src.nblk + b];
      t->smem = std::max(t->smem, dedisp_smem_bytes(fmt, cfg, cc, nww));
      int32_t* cg = t->crec.data() + g * t->g_crec;
      cg[((int64_t)src.nblk * src.nchan + b) * 2] = cc;
      cg[((int64_t)src.nblk * src.nchan + b) * 2 + 1] = nww;
      int32_t* cr = cg + (int64_t)b * src.nchan * 2;
      uint32_t* at = t->atab.data() + g * t->g_atab + b * t->atab_blk;
      const int nchunks = (src.nchan + cc - 1) / cc;
      for (int c = 0; c < nchunks * cc; ++c) {
        const int cl = c % cc;
        uint32_t* a = at + (int64_t)(c / cc) * B * cc + cl;
        if (c >= src.nchan) {
          // the zeroed landing window of an absent channel
          const uint32_t zero = (uint32_t)(cl * (nww + 4)) * 4u;
          for (int i = 0; i < B; ++i) a[(int64_t)i * cc] = zero;
          continue;
        }
        int64_t woff, span;
        window(dl, d0, d1, c, &woff, &span);
        for (int i = 0; i < B; ++i) {
          const int d = std::min(d0 + i, d1 - 1);
          const int64_t o = (int64_t)kPad + dl[(int64_t)d * src.dstride + c] - woff * spw;
          const int64_t om = o / spw;
          const int64_t kap = o % spw;
          // the unshifted copy is the landing window; copy kap >= 1 follows
          // the chunk's cc landing windows
          a[(int64_t)i * cc] =
              (uint32_t)(kap == 0 ? (cl * (nww + 4) + om) * 4
                                  : ((int64_t)cc * (nww + 4) + (cl * (spw - 1) + kap - 1) * nww + om) * 4);
        }
        cr[2 * c] = (int32_t)woff;
        cr[2 * c + 1] = (int32_t)span;
        // a copy reads at most span + 7 words from woff
        t->reach = std::max<int64_t>(t->reach, woff + span + 8);
      }
    }
  }
  return DD_OK;
}

std::shared_ptr<StageTab> stage_tab(Plan& p, int kind, const TabSrc& src, int fmt, int cfg,
                                    int cc_cap, int nww_uniform, bool upload, dd_status* err) {
  constexpr size_t kMaxTabs = 16;
  const std::array<int, 7> key = {kind, cfg, fmt, cc_cap, src.lo, nww_uniform, src.nblk};
  std::shared_ptr<StageTab> t;
  auto it = p.tabs.find(key);
  if (it != p.tabs.end()) {
    t = it->second;
  } else {
    t = std::make_shared<StageTab>();
    *err = build_stage_tab(src, fmt, cfg, cc_cap, nww_uniform, t.get());
    if (*err != DD_OK) return nullptr;
    if (p.tabs.size() < kMaxTabs) {
      p.tabs.emplace(key, t);
    } else if (upload) {
      // Full: drop the cache's references.  A table still held elsewhere (a
      // captured graph) lives on; the rest are freed here, which
      // synchronises the device, so no launch in flight still reads them.
      p.tabs.clear();
      p.tabs.emplace(key, t);
    }
    // else: a host-only caller (no device allocation or free allowed) takes
    // the table alone and the cache is left as it is
  }
  if (upload && !t->uploaded) {
    cudaError_t e = t->d_atab.ensure(t->atab.size() * 4);
    if (e == cudaSuccess)
      e = cudaMemcpy(t->d_atab.p, t->atab.data(), t->atab.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = t->d_crec.ensure(t->crec.size() * 4);
    if (e == cudaSuccess)
      e = cudaMemcpy(t->d_crec.p, t->crec.data(), t->crec.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      *err = cuda_status(e);
      return nullptr;
    }
    t->uploaded = true;
  }
  *err = DD_OK;
  return t;
}

void drop_stage_tabs(Plan& p, int kind_mask) {
  for (auto it = p.tabs.begin(); it != p.tabs.end();) {
    if (kind_mask & (1 << it->first[0]))
      it = p.tabs.erase(it);
    else
      ++it;
  }
}

// Bytes per output element of a launch, and whether every output row and
// tile start is 16-byte aligned (vector stores).
int out_elem_bytes(const Plan& p, int outk) {
  return outk == OUT_U32 && p.out_bits < 32 ? p.out_bits / 8 : 4;
}
bool out_vec_ok(const void* out, int64_t stride_elems, int esz) {
  return !(reinterpret_cast<uintptr_t>(out) & 15) && !((stride_elems * esz) & 15);
}

// Time tiles per work item.  An item of one or two chunks (the 32 channels of
// a sub-band stage) spends most of its time starting: the item counter, the
// block bounds, geometry and window records, then the first chunk's copy,
// one dependent latency after another.  Such items cover up to eight
// consecutive tiles of their trial block (four for two-chunk items), staged
// as one stream of chunks, so that start is paid once per group of tiles;
// the grid keeps at least eight items per SM.  On the survey band's sub-band
// stages (2^19 samples) groups of 4 / 8 / 16 tiles took 1.16 / 1.10 / 1.09 ms
// (stage 1) and 1.56 / 1.55 / 1.57 ms (stage 2).
static int tiles_per_item_for(const Plan& p, int nchan, int cc_cap, int64_t tiles,
                              int64_t items_per_tile) {
  const int chunks = (nchan + cc_cap - 1) / cc_cap;
  int r = chunks <= 1 ? 8 : (chunks == 2 ? 4 : 1);
  const int64_t want = 8 * (int64_t)std::max(1, p.num_sms);
  while (r > 1 && ((tiles + r - 1) / r) * items_per_tile < want) r >>= 1;
  return r;
}

// Fill launch parameters for a set of segments sharing one staged format.
// tune: the launch's tiling (words per lane resolved, see tuning_for).
static dd_status finish_launch(Plan& p, const Tuning& tune, int fmt, int outk, int vmax,
                               std::vector<SegSpec>& specs, bool vec_out, LaunchPlan* L) {
  const int cfg = tile_cfg_index(tune);
  const int B = kTileCfgs[cfg].nwarp * kTileCfgs[cfg].dpw;
  const int T = time_tile(fmt, tune);
  // 16 words a lane is compiled only for one or two samples a word
  if (kTileCfgs[cfg].k > 8 && fmt_spw(fmt) > 2) return DD_ERR_INVALID_ARG;
  int nchan_max = 0;
  for (auto& s : specs) nchan_max = std::max(nchan_max, (int)s.seg.nchan);
  // largest channels per chunk (the staging tables pick each block's own)
  int cc_cap = 4;
  while (cc_cap * 2 <= tune.chans_per_chunk) cc_cap *= 2;

  bool wide;
  int f0, f1, f2;
  flush_periods(fmt, vmax, nchan_max, &wide, &f0, &f1, &f2);
  // items of several time tiles where the multi-tile kernel is compiled for
  // the launch's kernel (scaled output runs the OUT_NARROW kernel)
  const int outk_run = outk == OUT_U32 && p.out_bits < 32 ? OUT_NARROW : outk;
  const bool mt_ok = multi_tile_compiled(fmt, outk_run, wide, cfg);
  // the 8-bit-lane sub-band stages have the multi-tile kernel only
  const bool mt_only = multi_tile_only(fmt, outk_run);
  if (mt_only && !mt_ok) return DD_ERR_INVALID_ARG;

  L->fmt = fmt;
  L->outk = outk;
  L->cfg = cfg;
  L->segs.clear();
  int64_t items = 0;
  bool multi = false;
  for (auto& s : specs) {
    Seg g = s.seg;
    if (g.n_groups < 1) g.n_groups = 1;
    if (g.ndm_last <= 0) g.ndm_last = g.ndm;
    if (g.ndm <= 0 || g.nsamps <= 0) continue;
    if (!g.blk) g.n_dmblk = (g.ndm + B - 1) / B;
    const int64_t tiles = (g.nsamps + T - 1) / T;
    g.tile0 = 0;
    g.tile_end = tiles;
    g.tiles_per_item =
        mt_ok ? tiles_per_item_for(p, g.nchan, cc_cap, tiles, (int64_t)g.n_dmblk * g.n_groups) : 1;
    multi = multi || g.tiles_per_item > 1;
    g.item_begin = items;
    items += (int64_t)g.n_dmblk * g.n_groups * ((tiles + g.tiles_per_item - 1) / g.tiles_per_item);
    L->segs.push_back(g);
  }
  if (L->segs.size() > (size_t)kMaxSegs) return DD_ERR_INVALID_ARG;
  if (outk == OUT_HALFIMG && (wide || (int64_t)nchan_max * std::max(vmax, 1) > 65535))
    return DD_ERR_OVERFLOW;
  if (outk == OUT_BYTEIMG && (wide || (int64_t)nchan_max * std::max(vmax, 1) > 127))
    return DD_ERR_OVERFLOW;
  if (fmt == FMT_SB8 && (wide || 2 * (int64_t)std::max(vmax, 1) > 255)) return DD_ERR_OVERFLOW;
  L->wide = wide;
  LaunchParams& lp = L->lp;
  std::memset(&lp, 0, sizeof(lp));
  lp.n_segs = (int32_t)L->segs.size();
  for (size_t i = 0; i < L->segs.size(); ++i) lp.segs[i] = L->segs[i];
  lp.f0 = f0;
  lp.f1 = f1;
  lp.f2 = f2;
  lp.n_items = items;
  lp.multi_tile = (multi || mt_only) ? 1 : 0;
  lp.vec_out = vec_out ? 1 : 0;
  // scaled low-bit output (Sec. 4.3): keep the top out_bits of the range a
  // sum can reach, nchan * vmax
  lp.out_bits = 32;
  lp.out_shift = 0;
  if (outk == OUT_U32 && p.out_bits < 32) {
    const uint64_t top = (uint64_t)std::max(nchan_max, 1) * (uint64_t)std::max(vmax, 1);
    int bl = 0;
    while (bl < 64 && (top >> bl) != 0) ++bl;
    lp.out_bits = p.out_bits;
    lp.out_shift = std::max(0, bl - p.out_bits);
    L->outk = OUT_NARROW;
  }
  // staging tables of each segment; shared memory for the widest block.  If
  // every block of every segment has one geometry, the kernel takes it from
  // the launch parameters.
  size_t smem = 0;
  bool uniform = true;
  int ucc = 0, unww = 0;
  {
    size_t i = 0;
    for (auto& sp : specs) {
      if (sp.seg.ndm <= 0 || sp.seg.nsamps <= 0) continue;
      dd_status err;
      std::shared_ptr<StageTab> t =
          stage_tab(*sp.owner, sp.kind, sp.src, fmt, cfg, cc_cap, window_words(fmt, tune, sp.spread),
                    !sp.no_upload, &err);
      if (!t) return err;
      // the kernel finds a block's geometry after the group's nblk x nchan
      // window records
      if (lp.segs[i].n_dmblk != sp.src.nblk || lp.segs[i].nchan != sp.src.nchan)
        return DD_ERR_INVALID_ARG;
      if (!t->uniform || (ucc && (t->cc != ucc || t->nww != unww))) uniform = false;
      ucc = t->cc;
      unww = t->nww;
      sp.tab = t;
      Seg& g = lp.segs[i];
      g.atab = sp.no_upload ? nullptr : static_cast<const uint32_t*>(t->d_atab.p);
      g.crec = sp.no_upload ? nullptr : static_cast<const int32_t*>(t->d_crec.p);
      g.g_atab = t->g_atab;
      g.g_crec = t->g_crec;
      g.atab_blk = t->atab_blk;
      L->segs[i] = g;
      smem = std::max(smem, t->smem);
      ++i;
    }
  }
  L->smem = smem;
  lp.per_block_geo = uniform ? 0 : 1;
  lp.cc = uniform ? ucc : 0;
  lp.nww = uniform ? unww : 0;
  int per_sm = 0;
  cudaError_t e = dedisp_max_blocks_per_sm(fmt, L->outk, wide, cfg, lp.per_block_geo != 0,
                                           lp.multi_tile != 0, L->smem, &per_sm);
  if (e != cudaSuccess) return cuda_status(e);
  if (per_sm < 1) return DD_ERR_INVALID_ARG;
  const int64_t resident = (int64_t)per_sm * std::max(1, p.num_sms);
  L->grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, resident));
  return DD_OK;
}

dd_status run_launch(Plan& p, LaunchPlan& L, cudaStream_t st, int timer_kind) {
  if (L.lp.n_items == 0) return DD_OK;
  L.lp.status = static_cast<uint32_t*>(p.d_status.p);
  L.lp.next_item = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(p.d_status.p) + 8 +
                                                         8 * (p.launch_seq++ % kItemCounters));
  cudaError_t e0 = cudaMemsetAsync(L.lp.next_item, 0, 8, st);
  if (e0 != cudaSuccess) return cuda_status(e0);
  KernelTimer kt(&p, timer_kind, st);
  return cuda_status(launch_dedisp(L.fmt, L.outk, L.wide, L.cfg, L.lp, L.grid, L.smem, st));
}

dd_status plan_direct_launch(Plan& p, int fmt, int outk, int vmax,
                             const std::vector<DirectJob>& jobs, LaunchPlan* L,
                             std::vector<std::shared_ptr<StageTab>>* tabs) {
  const int cfg = tile_cfg_index(tuning_for(p.tune, fmt));
  const int B = kTileCfgs[cfg].nwarp * kTileCfgs[cfg].dpw;
  std::vector<SegSpec> specs;
  bool vec = true;
  for (const DirectJob& j : jobs) {
    SegSpec s;
    std::memset(&s, 0, sizeof(s));
    const int bi = b_index(B);
    int32_t lo = j.plan->lo_B[bi];
    s.spread = j.plan->spread_B[bi];
    s.seg.blk = j.blk_dev ? j.blk_dev : static_cast<const int32_t*>(j.plan->d_blk[bi].p);
    s.seg.n_dmblk = (int32_t)j.plan->blocks_B[bi].size() - 1;
    if (!s.seg.blk) return DD_ERR_INVALID_ARG;
    s.seg.img = j.img;
    s.seg.delays = j.d_delays;
    s.seg.out = j.out;
    s.seg.row_words = j.row_words;
    s.seg.out_stride = j.out_stride;
    s.seg.nsamps = j.nsamps;
    s.seg.delay_stride = j.nchans;
    s.seg.nchan = j.nchans;
    s.seg.ndm = j.ndm;
    s.seg.lo_slack = lo;
    s.seg.n_groups = 1;
    s.seg.ndm_last = j.ndm;
    if (lo > kPad) return DD_ERR_INVALID_ARG;
    if (!out_vec_ok(j.out, j.out_stride, out_elem_bytes(p, outk))) vec = false;
    s.kind = 0;
    s.owner = const_cast<Plan*>(j.plan);
    const std::vector<int32_t>& bl = j.plan->blocks_B[bi];
    s.src = TabSrc{j.plan->delays.data(), 0, j.nchans, j.nchans, 1, bl.data(),
                   (int)bl.size() - 1, lo};
    s.no_upload = j.no_upload;
    specs.push_back(s);
  }
  dd_status st = finish_launch(p, tuning_for(p.tune, fmt), fmt, outk, vmax, specs, vec, L);
  if (st == DD_OK && tabs) {
    tabs->clear();
    for (auto& sp : specs) tabs->push_back(sp.tab);
  }
  return st;
}

// Geometry of the staged input image for a direct job: large enough for
// every compiled tile shape, so an image staged under one plan's tiling can
// be dedispersed by a launch that uses another's (batches).
static int64_t direct_row_words(Plan& p, int fmt, int64_t nsamps) {
  int64_t rw = 0;
  for (int i = 0; i < kNumTileCfgs; ++i) {
    Tuning t;
    t.dms_per_block = kTileCfgs[i].nwarp * kTileCfgs[i].dpw;
    t.words_per_lane = kTileCfgs[i].k;
    const int32_t spread = p.spread_B[b_index(t.dms_per_block)];
    rw = std::max(rw, image_row_words(fmt, t, nsamps, p.max_delay, spread));
  }
  return rw;
}

// Best-effort check that a device buffer holds `bytes` from `ptr`, through
// the driver's cuMemGetAddressRange (resolved at run time so that the library
// also loads on hosts without a driver).  Unknown ranges pass.
typedef int (*GetRangeFn)(unsigned long long*, size_t*, unsigned long long);
static GetRangeFn get_range_fn() {
  static GetRangeFn fn = [] {
    void* h = dlopen("libcuda.so.1", RTLD_LAZY | RTLD_NOLOAD);
    if (!h) h = dlopen("libcuda.so.1", RTLD_LAZY);
    if (!h) return (GetRangeFn) nullptr;
    void* f = dlsym(h, "cuMemGetAddressRange_v2");
    return (GetRangeFn)f;
  }();
  return fn;
}

static bool device_range_ok(const void* ptr, size_t bytes) {
  GetRangeFn fn = get_range_fn();
  if (!fn) return true;
  unsigned long long base = 0;
  size_t size = 0;
  if (fn(&base, &size, (unsigned long long)(uintptr_t)ptr) != 0) return true;
  return (unsigned long long)(uintptr_t)ptr + bytes <= base + size;
}

// The staged image of a direct job for nsamps outputs: `image` grown as
// needed, the job's image fields filled; nothing launched.
static dd_status prepare_direct_image(Plan& p, int nbits, int64_t nsamps, DevBuf& image,
                                      DirectJob* j) {
  const int fmt = fmt_for_nbits(nbits, p.nchans);
  const int64_t rw = direct_row_words(p, fmt, nsamps);
  cudaError_t e = image.ensure((size_t)p.nchans * rw * 4);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t* img = static_cast<uint32_t*>(image.p);
  j->img = img;
  j->row_words = rw;
  j->img_row_samples = rw * fmt_spw(fmt);
  j->d_delays = static_cast<const int32_t*>(p.d_delays.p);
  j->h_delays = p.delays.data();
  j->nchans = p.nchans;
  j->ndm = ndm(p);
  j->nsamps = nsamps;
  j->plan = &p;
  return DD_OK;
}

// Corner-turn `rows` input rows into `image` (grown as needed); fills the
// staged-image fields of a direct job for nsamps outputs.
dd_status stage_direct_image(Plan& p, const void* in, int nbits, int64_t in_stride, int64_t rows,
                             int64_t nsamps, DevBuf& image, cudaStream_t st, DirectJob* j) {
  dd_status s = prepare_direct_image(p, nbits, nsamps, image, j);
  if (s != DD_OK) return s;
  KernelTimer kt(&p, 0, st);
  return cuda_status(launch_corner_turn(nbits, fmt_for_nbits(nbits, p.nchans),
                                        static_cast<const uint8_t*>(in), in_stride, 0, rows,
                                        p.nchans, static_cast<const uint8_t*>(p.d_mask.p),
                                        const_cast<uint32_t*>(j->img), j->row_words, 0,
                                        j->row_words, st));
}

static dd_status exec_direct(Plan& p, const ExecArgs& a, int fmt) {
  const int64_t rows = a.nsamps_out + p.max_delay;
  DirectJob j;
  dd_status s0 = stage_direct_image(p, a.in, a.in_nbits, a.in_row_stride, rows, a.nsamps_out,
                                    p.d_image, a.st, &j);
  if (s0 != DD_OK) return s0;
  j.out = a.out;
  j.out_stride = a.out_stride;
  LaunchPlan L;
  dd_status s = plan_direct_launch(p, fmt, fmt == FMT_F32 ? OUT_F32 : OUT_U32,
                                   vmax_for_nbits(a.in_nbits), {j}, &L);
  if (s != DD_OK) return s;
  return run_launch(p, L, a.st);
}

// Direct transform from and into host memory.  The time tiles run as
// kOutParts launches, each over every trial block, so that the blocks of a
// tile still share its staged windows in L2 as in one launch (parts by
// trial block lose that reuse and ran 13 % slower in total).
//
// - Input: each part needs the image words its tiles' windows reach, which
//   need a prefix of the input rows.  Those rows are copied in on a second
//   stream piece by piece and corner-turned just before the part, so only
//   the first part waits for its rows; the rest arrive while it computes.
// - Output: each part's output columns, all rows, are copied to the host on
//   a third stream while the next part computes; the parts shrink towards
//   the end so that little copying is left once the last kernel ends.
//
// Synchronises.
static dd_status exec_direct_host_out(Plan& p, const ExecArgs& a, int fmt, const void* host_in,
                                      size_t in_bytes, void* host_out) {
  // part ends, in thousandths of the tiles
  constexpr int kOutParts = 8;
  static const int kPartEnd[kOutParts] = {160, 320, 480, 640, 800, 900, 960, 1000};
  dd_status s = ensure_device_tables(p);
  if (s != DD_OK) return s;
  const int64_t rows = a.nsamps_out + p.max_delay;
  DirectJob j;
  if ((s = prepare_direct_image(p, a.in_nbits, a.nsamps_out, p.d_image, &j)) != DD_OK) return s;
  j.out = a.out;
  j.out_stride = a.out_stride;
  LaunchPlan L;
  std::vector<std::shared_ptr<StageTab>> tabs;
  if ((s = plan_direct_launch(p, fmt, fmt == FMT_F32 ? OUT_F32 : OUT_U32,
                              vmax_for_nbits(a.in_nbits), {j}, &L, &tabs)) != DD_OK)
    return s;
  cudaError_t e = cudaSuccess;
  if (!p.copy_st) e = cudaStreamCreateWithFlags(&p.copy_st, cudaStreamNonBlocking);
  if (e == cudaSuccess && !p.in_st) e = cudaStreamCreateWithFlags(&p.in_st, cudaStreamNonBlocking);
  while (e == cudaSuccess && p.part_ev.size() < (size_t)(2 * kOutParts + 1)) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) p.part_ev.push_back(ev);
  }
  if (e != cudaSuccess) return cuda_status(e);
  const Seg g = L.lp.segs[0];
  const int spw = fmt_spw(fmt);
  const int64_t T = time_tile(fmt, tuning_for(p.tune, fmt));
  const int64_t tiles = (g.nsamps + T - 1) / T;
  const int64_t per_tile = (int64_t)g.n_groups * g.n_dmblk;
  const int64_t rw = j.row_words;
  const int64_t reach = tabs.empty() || !tabs[0] ? rw : tabs[0]->reach;
  const int esz = out_elem_bytes(p, fmt == FMT_F32 ? OUT_F32 : OUT_U32);
  const size_t pitch = (size_t)a.out_stride * esz;
  const size_t stride = (size_t)a.in_row_stride;
  uint8_t* const d_in = static_cast<uint8_t*>(const_cast<void*>(a.in));
  // the input stream starts after the caller's earlier work on a.st
  if ((e = cudaEventRecord(p.part_ev[2 * kOutParts], a.st)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(p.in_st, p.part_ev[2 * kOutParts], 0)) != cudaSuccess)
    return cuda_status(e);
  int64_t t0 = 0, w_done = 0, r_done = 0;
  for (int q = 0; q < kOutParts; ++q) {
    const int64_t t1 = tiles * kPartEnd[q] / 1000;
    if (t1 <= t0) continue;
    // image words this part's windows reach (whole 64-word pieces), and the
    // input rows those words are made from
    int64_t w_need = t1 >= tiles ? rw : std::min(rw, ((t1 * T / spw + reach + 63) / 64) * 64);
    if (w_need > w_done) {
      const int64_t r_need =
          w_need >= rw ? rows : std::min(rows, std::max<int64_t>(0, w_need * spw - kPad));
      if (r_need > r_done) {
        const size_t b0 = (size_t)r_done * stride;
        const size_t b1 = r_need >= rows ? in_bytes : std::min(in_bytes, (size_t)r_need * stride);
        if (b1 > b0 &&
            ((e = cudaMemcpyAsync(d_in + b0, static_cast<const uint8_t*>(host_in) + b0, b1 - b0,
                                  cudaMemcpyHostToDevice, p.in_st)) != cudaSuccess ||
             (e = cudaEventRecord(p.part_ev[kOutParts + q], p.in_st)) != cudaSuccess ||
             (e = cudaStreamWaitEvent(a.st, p.part_ev[kOutParts + q], 0)) != cudaSuccess))
          return cuda_status(e);
        r_done = r_need;
      }
      {
        KernelTimer kt(&p, 0, a.st);
        e = launch_corner_turn(a.in_nbits, fmt, d_in, a.in_row_stride, 0, rows, p.nchans,
                               static_cast<const uint8_t*>(p.d_mask.p),
                               const_cast<uint32_t*>(j.img), rw, w_done, w_need, a.st);
      }
      if (e != cudaSuccess) return cuda_status(e);
      w_done = w_need;
    }
    LaunchPlan Lq = L;
    const int rq = Lq.lp.segs[0].tiles_per_item;
    Lq.lp.segs[0].tile0 = t0;
    Lq.lp.segs[0].tile_end = t1;
    Lq.lp.n_items = ((t1 - t0 + rq - 1) / rq) * per_tile;
    Lq.grid = (int)std::min<int64_t>(L.grid, Lq.lp.n_items);
    if ((s = run_launch(p, Lq, a.st)) != DD_OK) return s;
    // output samples [t0 T, t1 T) of every trial are final: copy them out
    // (row-pitched: the caller's padding past nsamps is not written)
    const size_t c0 = (size_t)(t0 * T), c1 = (size_t)std::min<int64_t>(t1 * T, g.nsamps);
    if ((e = cudaEventRecord(p.part_ev[q], a.st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p.copy_st, p.part_ev[q], 0)) != cudaSuccess ||
        (e = cudaMemcpy2DAsync(static_cast<uint8_t*>(host_out) + c0 * esz, pitch,
                               static_cast<const uint8_t*>(a.out) + c0 * esz, pitch,
                               (c1 - c0) * esz, (size_t)ndm(p), cudaMemcpyDeviceToHost,
                               p.copy_st)) != cudaSuccess)
      return cuda_status(e);
    t0 = t1;
  }
  if ((e = cudaStreamSynchronize(a.st)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaStreamSynchronize(p.copy_st)) != cudaSuccess) return cuda_status(e);
  return DD_OK;
}

static dd_status exec_subband(Plan& p, const ExecArgs& a, int fmt) {
  if (fmt == FMT_F32) return DD_ERR_UNSUPPORTED_NBITS;
  // stage 1 writes the intermediate in 16-bit lanes (OUT_HALFIMG) from an
  // image of two samples a word: 8-bit input stays in 16-bit lanes here
  if (fmt == FMT_TRI) fmt = FMT_HALF;
  dd_status s = upload_subband(p);
  if (s != DD_OK) return s;
  const int C = p.nchans, Np = p.sb_chans, nsb = C / Np;
  const int n = ndm(p);
  const int ng = (n + p.sb_dms - 1) / p.sb_dms;
  const int vmax_in = vmax_for_nbits(a.in_nbits);
  const int64_t G = a.nsamps_out;
  const int64_t len1 = G + p.sb_len1_extra;  // stage-1 outputs per row

  // both stages run the plan's tiling (a 16-trial block for stage 1, which
  // pads the ng nominal DMs less, measured slower: 1.94 against 1.61 ms on
  // the survey gulp)
  const Tuning t1 = tuning_for(p.tune, fmt);
  const int B1 = t1.dms_per_block;
  const Tuning t2 = tuning_for(p.tune, fmt);
  const int B = t2.dms_per_block;

  // stage-1 geometry over the relative-delay table (ng x C, per sub-band)
  const int bi1 = b_index(B1);
  const int32_t spread1 = p.sb1_spread_B[bi1], lo1 = p.sb1_lo_B[bi1];
  const int32_t maxrel = p.sb_maxrel;
  if (lo1 > kPad) return DD_ERR_INVALID_ARG;
  const int64_t rw = image_row_words(fmt, t1, len1, maxrel, spread1);
  cudaError_t e = p.d_image.ensure((size_t)C * rw * 4);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t* img = static_cast<uint32_t*>(p.d_image.p);
  const int64_t rows = G + p.sb_max_delay;
  {
    KernelTimer kt(&p, 0, a.st);
    e = launch_corner_turn(a.in_nbits, fmt, static_cast<const uint8_t*>(a.in), a.in_row_stride, 0,
                           rows, C, static_cast<const uint8_t*>(p.d_mask.p), img, rw, 0, rw,
                           a.st);
  }
  if (e != cudaSuccess) return cuda_status(e);

  // intermediate: 8-bit image rows when stage-1 sums stay below 128 (1- and
  // 2-bit input; stage 2 then adds two sub-bands a lane and a trial's total
  // fits 16 bits), else 16-bit rows when they fit, else 32-bit.  The 8-bit
  // stages exist as multi-tile kernels of the default tiles only (stage 1:
  // 32 trials, 4 words a lane; stage 2: 32 trials, 8 words a lane) and for
  // uint32 output rows.
  const int64_t vmax1 = (int64_t)Np * vmax_in;
  const bool byte =
      fmt == FMT_NIB && vmax1 <= 127 && (int64_t)C * vmax_in <= 65535 && p.out_bits == 32 &&
      multi_tile_compiled(FMT_NIB, OUT_BYTEIMG, false, tile_cfg_index(t1)) &&
      multi_tile_compiled(FMT_SB8, OUT_U32, false, tile_cfg_index(tuning_for(p.tune, FMT_SB8)));
  const bool half = !byte && vmax1 <= 65535;
  const int fmt2 = byte ? FMT_SB8 : (half ? FMT_HALF : FMT_U32);
  const int bi = b_index(B);
  const int32_t spread2 = p.sb2_spread_B[bi], lo2 = p.sb2_lo_B[bi];
  if (lo2 > kPad) return DD_ERR_INVALID_ARG;
  const int T1 = time_tile(fmt, t1);
  const int spw2 = fmt_spw(fmt2);
  int64_t rw2 = image_row_words(fmt2, tuning_for(p.tune, fmt2), G, (int32_t)p.sb_len1_extra, spread2);
  const int64_t st1_words = (kPad + ((len1 + T1 - 1) / T1) * T1) / spw2 + 8;
  rw2 = std::max(rw2, (st1_words + 31) & ~(int64_t)31);
  const size_t s_bytes = (size_t)ng * nsb * rw2 * 4;
  if (p.d_sb_S.bytes < s_bytes || !p.d_sb_S.p) {
    if ((e = p.d_sb_S.ensure(s_bytes)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(p.d_sb_S.p, 0, p.d_sb_S.bytes, a.st)) != cudaSuccess)
      return cuda_status(e);
  }
  uint32_t* S = static_cast<uint32_t*>(p.d_sb_S.p);

  // stage 1: sub-band n (a group of the segment) sums its N' channels at
  // each trial group's nominal DM
  std::vector<SegSpec> specs(1);
  {
    SegSpec& sp = specs[0];
    std::memset(&sp, 0, sizeof(sp));
    sp.spread = spread1;
    Seg& g = sp.seg;
    g.img = img;
    g.row_words = rw;
    g.delays = static_cast<const int32_t*>(p.d_sb_rel.p);
    g.delay_stride = C;
    g.nchan = Np;
    g.ndm = ng;
    g.ndm_last = ng;
    g.n_groups = nsb;
    g.g_img = (int64_t)Np * rw;
    g.g_delay = Np;
    g.g_out = rw2;
    g.lo_slack = lo1;
    g.blk = static_cast<const int32_t*>(p.d_sb1_blk[bi1].p);
    g.n_dmblk = p.sb1_nblk_B[bi1];
    g.nsamps = len1;
    g.out = S + kPad / spw2;
    g.out_stride = (int64_t)nsb * rw2;
    sp.kind = 1;
    sp.owner = &p;
    sp.src = TabSrc{p.sb_rel.data(), Np, C, Np, nsb, p.sb1_blk_B[bi1].data(), p.sb1_nblk_B[bi1],
                    lo1};
  }
  LaunchPlan L1;
  s = finish_launch(p, t1, fmt, byte ? OUT_BYTEIMG : (half ? OUT_HALFIMG : OUT_U32), vmax_in,
                    specs, true, &L1);
  if (s != DD_OK) return s;
  if ((s = run_launch(p, L1, a.st)) != DD_OK) return s;

  // stage 2: each trial sums the sub-bands of its group (a group of the
  // segment), shifted by delay(d, nN')
  {
    SegSpec& sp = specs[0];
    std::memset(&sp, 0, sizeof(sp));
    sp.spread = spread2;
    Seg& q = sp.seg;
    q.img = S;
    q.row_words = rw2;
    q.delays = static_cast<const int32_t*>(p.d_sb_d2.p);
    q.delay_stride = nsb;
    q.nchan = nsb;
    q.ndm = p.sb_dms;
    q.ndm_last = n - (ng - 1) * p.sb_dms;
    q.n_groups = ng;
    q.g_img = (int64_t)nsb * rw2;
    q.g_delay = p.sb_dms * nsb;
    q.g_out = (int64_t)p.sb_dms * a.out_stride;
    q.lo_slack = lo2;
    q.blk = static_cast<const int32_t*>(p.d_sb2_blk[bi].p);
    q.n_dmblk = p.sb2_nblk_B[bi];
    q.nsamps = G;
    q.out = a.out;
    q.out_stride = a.out_stride;
    sp.kind = 2;
    sp.owner = &p;
    sp.src = TabSrc{p.sb_d2.data(), (int64_t)p.sb_dms * nsb, nsb, nsb, ng,
                    p.sb2_blk_B[bi].data(), p.sb2_nblk_B[bi], lo2};
  }
  const bool vec = out_vec_ok(a.out, a.out_stride, out_elem_bytes(p, OUT_U32));
  LaunchPlan L2;
  s = finish_launch(p, tuning_for(p.tune, fmt2), fmt2, OUT_U32, (int)std::min<int64_t>(vmax1, INT_MAX),
                    specs, vec, &L2);
  if (s != DD_OK) return s;
  return run_launch(p, L2, a.st, DD_KERNEL_STAGE2);
}

dd_status exec_device(Plan& p, const ExecArgs& a) {
  const int fmt = fmt_for_nbits(a.in_nbits, p.nchans);
  if (fmt < 0) return DD_ERR_UNSUPPORTED_NBITS;
  dd_status s = ensure_device_tables(p);
  if (s != DD_OK) return s;
  if (a.tree) return exec_tree(p, a);
  return a.subband ? exec_subband(p, a, fmt) : exec_direct(p, a, fmt);
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_execute(dd_plan plan, int64_t nsamps_out, const void* in, int in_nbits,
                                int64_t in_row_stride, void* out, int64_t out_stride,
                                void* cuda_stream, unsigned flags) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !in || !out || nsamps_out <= 0 || out_stride < nsamps_out) return DD_ERR_INVALID_ARG;
  const int fmt = fmt_for_nbits(in_nbits, p->nchans);
  if (fmt < 0) return DD_ERR_UNSUPPORTED_NBITS;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  const int64_t row_bytes =
      in_nbits == 32 ? (int64_t)p->nchans * 4 : ((int64_t)p->nchans * in_nbits + 7) / 8;
  if (in_row_stride < row_bytes) return DD_ERR_INVALID_ARG;
  const bool sub = (flags & DD_SUBBAND) != 0;
  const bool scr = (flags & DD_SCRUNCH) != 0;
  const bool tree = (flags & DD_TREE) != 0;
  if (sub && p->sb_chans <= 0) return DD_ERR_INVALID_ARG;
  if (scr && (sub || p->scrunch_max <= 0 || !(flags & DD_DEVICE_PTRS)))
    return DD_ERR_INVALID_ARG;
  if (scr && in_nbits > 4) return DD_ERR_UNSUPPORTED_NBITS;
  if (tree && (sub || scr || p->tree_chans <= 0 || p->out_bits != 32)) return DD_ERR_INVALID_ARG;
  if (tree && in_nbits == 32) return DD_ERR_UNSUPPORTED_NBITS;
  std::lock_guard<std::mutex> lk(p->mu);
  if (sub) {
    dd_status s = prepare_subband(*p);
    if (s != DD_OK) return s;
  }
  if (scr) {
    dd_status s = prepare_scrunch(*p);
    if (s != DD_OK) return s;
  }
  if (tree) {
    dd_status s = prepare_tree(*p);
    if (s != DD_OK) return s;
  }
  const int64_t rows = scr    ? scrunch_input_rows(*p, nsamps_out)
                       : tree ? nsamps_out + tree_input_extra(*p)
                              : nsamps_out + (sub ? p->sb_max_delay : p->max_delay);
  ExecArgs a;
  a.nsamps_out = nsamps_out;
  a.in_nbits = in_nbits;
  a.in_row_stride = in_row_stride;
  a.in_rows = rows;
  a.out_stride = out_stride;
  a.st = static_cast<cudaStream_t>(cuda_stream);
  a.subband = sub;
  a.tree = tree;
  const size_t in_bytes = (size_t)(rows - 1) * in_row_stride + row_bytes;
  const int esz = p->out_bits / 8;
  if (esz != 4 && (in_nbits == 32 || scr)) return DD_ERR_INVALID_ARG;
  const size_t out_bytes = (size_t)((int64_t)(ndm(*p) - 1) * out_stride + nsamps_out) * esz;
  if (flags & DD_DEVICE_PTRS) {
    if (!device_range_ok(in, in_bytes)) return DD_ERR_INPUT_TOO_SHORT;
    if (!device_range_ok(out, out_bytes)) return DD_ERR_INVALID_ARG;
    a.in = in;
    a.out = out;
    return scr ? exec_scrunch(*p, a) : exec_device(*p, a);
  }
  // host pointers: stage through plan-owned device buffers
  cudaError_t e;
  if ((e = p->d_in.ensure(in_bytes)) != cudaSuccess) return cuda_status(e);
  if ((e = p->d_out.ensure(out_bytes)) != cudaSuccess) return cuda_status(e);
  a.in = p->d_in.p;
  a.out = p->d_out.p;
  if (!sub && !tree) return exec_direct_host_out(*p, a, fmt, in, in_bytes, out);
  if ((e = cudaMemcpyAsync(p->d_in.p, in, in_bytes, cudaMemcpyHostToDevice, a.st)) != cudaSuccess)
    return cuda_status(e);
  dd_status s = exec_device(*p, a);
  if (s != DD_OK) return s;
  if ((e = cudaMemcpy2DAsync(out, (size_t)out_stride * esz, p->d_out.p,
                             (size_t)out_stride * esz, (size_t)nsamps_out * esz,
                             (size_t)ndm(*p), cudaMemcpyDeviceToHost, a.st)) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaStreamSynchronize(a.st)) != cudaSuccess) return cuda_status(e);
  return DD_OK;
}

extern "C" dd_status dd_plan_set_output_bits(dd_plan plan, int bits) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || (bits != 8 && bits != 16 && bits != 32)) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(p->mu);
  p->out_bits = bits;
  return DD_OK;
}

extern "C" dd_status dd_plan_get_chunk_geometry(dd_plan plan, int in_nbits, int32_t* n_blocks,
                                               int32_t* chans_per_chunk, int32_t* nww_out,
                                               size_t* smem_bytes) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !n_blocks) return DD_ERR_INVALID_ARG;
  const int fmt = fmt_for_nbits(in_nbits, p->nchans);
  if (fmt < 0) return DD_ERR_UNSUPPORTED_NBITS;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  std::lock_guard<std::mutex> lk(p->mu);
  const Tuning t = tuning_for(p->tune, fmt);
  const int cfg = tile_cfg_index(t);
  const int bi = b_index(kTileCfgs[cfg].nwarp * kTileCfgs[cfg].dpw);
  const std::vector<int32_t>& bl = p->blocks_B[bi];
  const int nblk = (int)bl.size() - 1;
  *n_blocks = nblk;
  if (!chans_per_chunk && !nww_out && !smem_bytes) return DD_OK;
  int cc_cap = 4;
  while (cc_cap * 2 <= p->tune.chans_per_chunk) cc_cap *= 2;
  const TabSrc src{p->delays.data(), 0, p->nchans, p->nchans, 1, bl.data(), nblk, p->lo_B[bi]};
  dd_status err;
  std::shared_ptr<StageTab> tab =
      stage_tab(*p, 0, src, fmt, cfg, cc_cap, window_words(fmt, t, p->spread_B[bi]), false, &err);
  if (!tab) return err;
  for (int b = 0; b < nblk; ++b) {
    const int32_t* geo = tab->crec.data() + ((int64_t)nblk * p->nchans + b) * 2;
    if (chans_per_chunk) chans_per_chunk[b] = geo[0];
    if (nww_out) nww_out[b] = geo[1];
  }
  if (smem_bytes) *smem_bytes = tab->smem;
  return DD_OK;
}

extern "C" dd_status dd_plan_get_input_rows(dd_plan plan, int64_t nsamps_out, unsigned flags,
                                           int64_t* rows) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !rows || nsamps_out < 0) return DD_ERR_INVALID_ARG;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  std::lock_guard<std::mutex> lk(p->mu);
  if (flags & DD_SCRUNCH) {
    if (p->scrunch_max <= 0) return DD_ERR_INVALID_ARG;
    dd_status s = prepare_scrunch(*p);
    if (s != DD_OK) return s;
    *rows = scrunch_input_rows(*p, nsamps_out);
  } else if (flags & DD_SUBBAND) {
    if (p->sb_chans <= 0) return DD_ERR_INVALID_ARG;
    dd_status s = prepare_subband(*p);
    if (s != DD_OK) return s;
    *rows = nsamps_out + p->sb_max_delay;
  } else if (flags & DD_TREE) {
    if (p->tree_chans <= 0) return DD_ERR_INVALID_ARG;
    dd_status s = prepare_tree(*p);
    if (s != DD_OK) return s;
    *rows = nsamps_out + tree_input_extra(*p);
  } else {
    *rows = nsamps_out + p->max_delay;
  }
  return DD_OK;
}

extern "C" dd_status dd_probe_int_add(int64_t adds_per_thread, void* cuda_stream,
                                      double* adds_per_second, double* kernel_ms) {
  if (adds_per_thread < 32 || !adds_per_second) return DD_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, sms) * 8;
  const int64_t iters = (adds_per_thread / 8 / 4) * 4;
  uint32_t* seed = nullptr;
  uint32_t* sink = nullptr;
  cudaError_t e = cudaMalloc(&seed, 16 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)grid * 256 * 4);
  if (e != cudaSuccess) {
    cudaFree(seed);
    return cuda_status(e);
  }
  uint32_t h[16];
  for (int i = 0; i < 16; ++i) h[i] = 0x9E3779B9u * (i + 1);
  cudaEvent_t a = nullptr, b = nullptr;
  float ms = 0.f;
  e = cudaMemcpy(seed, h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = launch_probe(seed, iters, sink, grid, st);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) e = launch_probe(seed, iters, sink, grid, st);
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(seed);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_status(e);
  const double adds = (double)grid * 256.0 * (double)iters * 8.0;
  *adds_per_second = adds / (ms * 1e-3);
  if (kernel_ms) *kernel_ms = ms;
  return DD_OK;
}
