// Body of the direct dedispersion kernel, included twice by dd_dedisp.cuh:
// as k_dedisp (DD_MT 0: one time tile per work item) and as k_dedisp_mt
// (DD_MT 1: a work item covers Seg::tiles_per_item consecutive tiles of its
// trial block, staged as one stream of chunks, so that an item of one or two
// chunks pays its start once per group of tiles).  The one-tile kernel is
// kept free of the multi-tile bookkeeping: it is register-bound, and even
// compile-time-dead tile state changed its code.
//
// Expects DD_KERNEL (the kernel's name) and DD_MT (0 or 1) to be defined.
template <int FMT, int OUTK, bool WIDE, int NWARP, int DPW, int K, bool PBG>
__global__ void __launch_bounds__(NWARP * 32, (NWARP <= 8 ? 2 : 1)) DD_KERNEL(const LaunchParams p) {
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
  // FINE: the chunk size is any multiple of 4 (4- and 8-bit input: 8-bit and
  // 10-bit lanes); otherwise a power of two
  constexpr bool FINE = FMT == FMT_TRI || FMT == FMT_BYTE;
  struct Geo {
    int cc, cc_log, nww, nwl, buf_words, n_entries, tpc_log, bc;
    int tpc = 0, bq = 0;  // FINE: builder threads per channel, this thread's index among them
    uint32_t* s_addr;
  };
  auto make_geo = [&](int cc, int nww) {
    Geo g;
    g.cc = cc;  // power of two (FINE: multiple of 4), 4..32
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
    if constexpr (FINE) {
      // (the NT mod cc threads past the last channel build nothing)
      g.n_entries = B * cc;
      g.tpc = NT / cc;
      g.bc = tid / g.tpc;
      g.bq = tid - g.bc * g.tpc;
    }
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
#if DD_MT
    // the item's time tiles [tileA, tileB): consecutive tiles of one trial
    // block, staged as one stream of chunks
    const int64_t tileA = S.tile0 + lt * S.tiles_per_item;
    const int64_t tileB = min(tileA + (int64_t)S.tiles_per_item, S.tile_end);
#else
    const int64_t tile = S.tile0 + lt;
#endif
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
#if !DD_MT
    const int64_t t0 = tile * T;
    const int64_t t_end = min(t0 + T, S.nsamps);
#endif
    const int64_t row_words = S.row_words;
    const uint32_t* __restrict__ img = S.img + (int64_t)grp * S.g_img;
    uint32_t* const out_g = reinterpret_cast<uint32_t*>(S.out) + (int64_t)grp * S.g_out;
#if DD_MT
    if (nd <= 0 || tileA * T >= S.nsamps || tileB <= tileA) {
#else
    if (nd <= 0 || t0 >= S.nsamps) {
#endif
      if (tid == 0) atomicOr(p.status, DEV_BAD_ITEM);
      continue;
    }
    const Geo G = PBG ? make_geo(bgeo.x, bgeo.y) : geo_launch;
    const int cc = G.cc, cc_log = G.cc_log, nww = G.nww, nwl = G.nwl;
    uint32_t* const s_addr = G.s_addr;
    const int buf_words = G.buf_words;
    const int n_entries = G.n_entries, tpc_log = G.tpc_log, bc = G.bc;
    const int nchunks = FINE ? (nchan + cc - 1) / cc : (nchan + cc - 1) >> cc_log;
    const uint32_t* __restrict__ atab =
        S.atab + (int64_t)grp * S.g_atab + (int64_t)blk * S.atab_blk;
#if !DD_MT
    const int64_t t0w = t0 / SPW;  // image word of time t0 - kPad
#endif

    // window record of channel c0 + (warp 0: lane; builders: bc) of chunk k
    auto rec_of = [&](int k, int c) -> int2 {
      const int ca = (FINE ? k * cc : k << cc_log) + c;
      return ca < nchan ? __ldg(&crec[ca]) : make_int2(0, 32 * K);
    };
    // TMA of chunk k (warp 0): the offsets, then each channel's window.  A
    // window running past the end of its row (a launch over images of
    // different lengths) is shortened: those words are beyond every valid
    // output of this image.
#if DD_MT
    // t0w: image word of time t0 - kPad of the chunk's tile (t0 = tile * T)
    auto issue = [&](int k, int nb, int2 r, int64_t t0w) {
#else
    auto issue = [&](int k, int nb, int2 r) {
#endif
      const uint32_t bar = bar0 + 8u * nb;
      const int c0 = FINE ? k * cc : k << cc_log;
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
    if constexpr (FMT == FMT_TRI) paired = true;

    Acc<FMT, WIDE> acc[DPW][K];
#pragma unroll
    for (int i = 0; i < DPW; ++i)
#pragma unroll
      for (int j = 0; j < K; ++j) acc[i][j].zero();
    int g0 = 0, g1 = 0, g2 = 0;

    // prologue: chunk 0
    int2 rec_w = make_int2(0, 0);  // warp 0: window record of the next chunk to issue
#if DD_MT
    if (warp == 0) issue(0, kk & 1, rec_of(0, lane), tileA * (T / SPW));
#else
    if (warp == 0) issue(0, kk & 1, rec_of(0, lane));
#endif
    int span = COPIES ? rec_of(0, bc).y : 0;  // builders: words of this chunk's window

#if DD_MT
    // the item's tiles one after another; the next chunk (kn of its tile) is
    // staged while this one is summed, across tile boundaries too
    for (int64_t tt = tileA; tt < tileB; ++tt) {
    const bool last_tile = tt + 1 == tileB;
#endif
    for (int k = 0; k < nchunks; ++k, ++kk) {
      const int buf = kk & 1;
      const int c0 = FINE ? k * cc : k << cc_log;
#if DD_MT
      const bool tile_done = k + 1 == nchunks;
      const bool more = !tile_done || !last_tile;
      const int kn = tile_done ? 0 : k + 1;
#else
      const bool more = k + 1 < nchunks;
#endif
      int span_next = 0;
      if (more) {
#if DD_MT
        if (warp == 0) rec_w = rec_of(kn, lane);
        if (COPIES) span_next = rec_of(kn, bc).y;
#else
        if (warp == 0) rec_w = rec_of(k + 1, lane);
        if (COPIES) span_next = rec_of(k + 1, bc).y;
#endif
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
        const int nq = (!FINE || c < cc) ? (min(span, nww) + 3) >> 2 : 0;
        const bool live = c0 + c < nchan;
        const int q0 = FINE ? G.bq : tid & ((1 << tpc_log) - 1);
        const int qs = FINE ? G.tpc : 1 << tpc_log;
        for (int q = q0; q < nq; q += qs) {
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
#if DD_MT
      if (more && warp == 0) issue(kn, buf ^ 1, rec_w, (tile_done ? tt + 1 : tt) * (T / SPW));
#else
      if (more && warp == 0) issue(k + 1, buf ^ 1, rec_w);
#endif
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
            const uint32_t* const e =
                sa + (FINE ? (warp * DPW + i) * cc : (warp * DPW + i) << cc_log) + cg;
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
          // four groups (two pairs), then moves to its 32-bit sum
          auto moved = [&]() {
#pragma unroll
            for (int i = 0; i < DPW; ++i)
#pragma unroll
              for (int j = 0; j < K; ++j) acc[i][j].flush1();
          };
          int cg = 0;
          for (; cg + 16 <= cc; cg += 16) {
            pair8(cg);
            pair8(cg + 8);
            moved();
          }
          if (cg < cc) {
            // 4, 8 or 12 channels left: at most three groups, then the move
            if (cg + 8 <= cc) {
              pair8(cg);
              cg += 8;
            }
            if (cg < cc) {
              // one group of four channels
#pragma unroll
              for (int i = 0; i < DPW; ++i) {
                const uint4 a4 = *reinterpret_cast<const uint4*>(sa + (warp * DPW + i) * cc + cg);
                const uint32_t q0 = a4.x + lane_off, q1 = a4.y + lane_off;
                const uint32_t q2 = a4.z + lane_off, q3 = a4.w + lane_off;
#pragma unroll
                for (int j = 0; j < K; ++j)
                  acc[i][j].add4(lds32(q0 + 128u * j), lds32(q1 + 128u * j),
                                 lds32(q2 + 128u * j), lds32(q3 + 128u * j));
              }
            }
            moved();
          }
        }
      } else
      for (int cg = 0; cg < cc; cg += 4) {
#pragma unroll
        for (int i = 0; i < DPW; ++i) {
          const uint4 a4 = *reinterpret_cast<const uint4*>(
              sa + (FINE ? (warp * DPW + i) * cc : (warp * DPW + i) << cc_log) + cg);
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
#if DD_MT
    // tile tt is complete: its sums out below, then fresh sums for the next
    const int64_t t0 = tt * T;
    const int64_t t_end = min(t0 + T, S.nsamps);
#else
    // all warps are done with this item's buffers before the next prologue
    __syncthreads();
#endif

    // (d) exact sums out: u32 rows, float rows, or 16- or 8-bit image rows
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
        } else if constexpr (OUTK == OUT_BYTEIMG) {
          // stage-1 sums below 128 (the plan's check), four to a word
          static_assert(SPW == 8, "8-bit image rows come from the 4-bit lanes");
          uint32_t* dst = out_g + (int64_t)(d0 + slot) * S.out_stride + (tw >> 2);
          *reinterpret_cast<uint2*>(dst) =
              make_uint2(v[0] | (v[1 % SPW] << 8) | (v[2 % SPW] << 16) | (v[3 % SPW] << 24),
                         v[4 % SPW] | (v[5 % SPW] << 8) | (v[6 % SPW] << 16) | (v[7 % SPW] << 24));
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
#if DD_MT
#pragma unroll
    for (int i = 0; i < DPW; ++i)
#pragma unroll
      for (int j = 0; j < K; ++j) acc[i][j].zero();
    g0 = g1 = g2 = 0;
    }
    // all warps are done with this item's buffers before the next prologue
    __syncthreads();
#endif
  }
}
