// Streaming (consecutive gulps of one beam), batched multi-beam launches and
// the tiling autotuner.
//
// Eq. 2 needs input rows up to t + max_delay for output t, so a beam's series
// is processed gulp by gulp with the last max_delay input rows kept on the
// device: each push appends the gulp after that tail, dedisperses every output
// that became computable, and keeps the rows the next output will need.  The
// paper processes fixed one-minute blocks and has no streaming; this is the
// overlap that makes consecutive blocks equal one continuous transform.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>

#include "dd_internal.h"

namespace dd {

struct StreamState {
  Plan* plan = nullptr;
  int nbits = 0;
  int64_t row_bytes = 0;   // packed bytes per input row
  int64_t max_gulp = 0;
  int64_t cap_rows = 0;    // rows per raw buffer (max_delay + max_gulp)
  DevBuf raw[2];           // ping-pong raw input buffers, tail at the front
  int cur = 0;
  int64_t tail_rows = 0;   // valid rows at the front of raw[cur]
  int64_t samples_in = 0, samples_out = 0;
  DevBuf image;            // this stream's staged image
};

static int64_t input_row_bytes(int nchans, int nbits) {
  return nbits == 32 ? (int64_t)nchans * 4 : ((int64_t)nchans * nbits + 7) / 8;
}

// Append n rows (pitch in_stride) after the tail of raw[cur].
static dd_status append_rows(StreamState& s, const void* in, int64_t n, int64_t in_stride,
                             bool device, cudaStream_t st) {
  if (n == 0) return DD_OK;
  uint8_t* dst = static_cast<uint8_t*>(s.raw[s.cur].p) + s.tail_rows * s.row_bytes;
  const cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpy2DAsync(dst, s.row_bytes, in, in_stride, s.row_bytes, n, kind, st);
  return cuda_status(e);
}

// Keep rows [first, total) of raw[cur] as the new tail (moved to the front of
// the other buffer, so the copy never overlaps its source).
static dd_status keep_tail(StreamState& s, int64_t first, int64_t total, cudaStream_t st) {
  const int64_t keep = total - first;
  if (keep > 0 && first > 0) {
    const uint8_t* src = static_cast<const uint8_t*>(s.raw[s.cur].p) + first * s.row_bytes;
    cudaError_t e = cudaMemcpyAsync(s.raw[s.cur ^ 1].p, src, (size_t)keep * s.row_bytes,
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    s.cur ^= 1;
  }
  s.tail_rows = keep;
  return DD_OK;
}

// Stage one push: append the gulp and corner-turn [tail | gulp] into the
// stream's image.  Returns the outputs that became computable in *n_out and
// the total rows in *total.
static dd_status stream_stage(StreamState& s, const void* in, int64_t n_in, int64_t in_stride,
                              bool device, cudaStream_t st, DirectJob* job, int64_t* n_out,
                              int64_t* total) {
  Plan& p = *s.plan;
  dd_status r = append_rows(s, in, n_in, in_stride, device, st);
  if (r != DD_OK) return r;
  *total = s.tail_rows + n_in;
  *n_out = std::max<int64_t>(0, *total - p.max_delay);
  if (*n_out == 0) return DD_OK;
  return stage_direct_image(p, s.raw[s.cur].p, s.nbits, s.row_bytes, *total, *n_out, s.image, st,
                            job);
}

}  // namespace dd

using namespace dd;

struct dd_stream_s {
  StreamState s;
};

struct BatchItem {
  dd_stream stream;
  const void* in;
  int64_t n_in, in_stride;
  void* out;
  int64_t out_stride;
};

struct dd_batch_s {
  std::vector<BatchItem> items;
};

extern "C" {

dd_status dd_stream_create(dd_stream* out, dd_plan plan, int nbits, int64_t max_gulp) {
  if (!out) return DD_ERR_INVALID_ARG;
  *out = nullptr;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || max_gulp <= 0) return DD_ERR_INVALID_ARG;
  if (fmt_for_nbits(nbits, p->nchans) < 0) return DD_ERR_UNSUPPORTED_NBITS;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  if (p->out_bits != 32) return DD_ERR_INVALID_ARG;  // streams write uint32 rows
  dd_stream h = new (std::nothrow) dd_stream_s();
  if (!h) return DD_ERR_OOM;
  StreamState& s = h->s;
  s.plan = p;
  s.nbits = nbits;
  s.row_bytes = input_row_bytes(p->nchans, nbits);
  s.max_gulp = max_gulp;
  s.cap_rows = p->max_delay + max_gulp;
  for (int i = 0; i < 2; ++i) {
    cudaError_t e = s.raw[i].ensure((size_t)s.cap_rows * s.row_bytes);
    if (e != cudaSuccess) {
      delete h;
      return cuda_status(e);
    }
  }
  *out = h;
  return DD_OK;
}

void dd_stream_destroy(dd_stream h) { delete h; }

dd_status dd_stream_push(dd_stream h, const void* in, int64_t n_in, int64_t in_stride, void* out,
                         int64_t out_stride, int64_t* nsamps_out, void* cuda_stream,
                         unsigned flags) {
  if (!h || !in || !out || n_in < 0 || !nsamps_out) return DD_ERR_INVALID_ARG;
  StreamState& s = h->s;
  Plan& p = *s.plan;
  *nsamps_out = 0;
  if (n_in > s.max_gulp || in_stride < s.row_bytes || out_stride < n_in) return DD_ERR_INVALID_ARG;
  if (p.max_delay + s.max_gulp > s.cap_rows) return DD_ERR_INVALID_ARG;  // plan changed
  if (p.out_bits != 32) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(p.mu);
  dd_status r = ensure_device_tables(p);
  if (r != DD_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const bool device = (flags & DD_DEVICE_PTRS) != 0;
  const int fmt = fmt_for_nbits(s.nbits, p.nchans);
  DirectJob job;
  int64_t n_out = 0, total = 0;
  if ((r = stream_stage(s, in, n_in, in_stride, device, st, &job, &n_out, &total)) != DD_OK)
    return r;
  if (n_out > 0) {
    void* dout = out;
    if (!device) {
      const size_t ob = (size_t)((int64_t)(ndm(p) - 1) * out_stride + n_out) * 4;
      cudaError_t e = p.d_out.ensure(ob);
      if (e != cudaSuccess) return cuda_status(e);
      dout = p.d_out.p;
    }
    job.out = dout;
    job.out_stride = out_stride;
    LaunchPlan L;
    r = plan_direct_launch(p, fmt, fmt == FMT_F32 ? OUT_F32 : OUT_U32, vmax_for_nbits(s.nbits),
                           {job}, &L);
    if (r != DD_OK) return r;
    if ((r = run_launch(p, L, st)) != DD_OK) return r;
    if (!device) {
      cudaError_t e = cudaMemcpy2DAsync(out, out_stride * 4, dout, out_stride * 4, n_out * 4,
                                        ndm(p), cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return cuda_status(e);
    }
  }
  if ((r = keep_tail(s, n_out, total, st)) != DD_OK) return r;
  s.samples_in += n_in;
  s.samples_out += n_out;
  *nsamps_out = n_out;
  if (!device) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return DD_OK;
}

dd_status dd_stream_position(dd_stream h, int64_t* in, int64_t* out) {
  if (!h) return DD_ERR_INVALID_ARG;
  if (in) *in = h->s.samples_in;
  if (out) *out = h->s.samples_out;
  return DD_OK;
}

// Snapshot layout: 8 int64 header words (magic, nchans, nbits, row_bytes,
// samples_in, samples_out, tail_rows, max_delay) then the tail rows.
static const int64_t kSnapMagic = 0x44445354524d3031LL;

dd_status dd_stream_snapshot_size(dd_stream h, int64_t* bytes) {
  if (!h || !bytes) return DD_ERR_INVALID_ARG;
  *bytes = 64 + h->s.tail_rows * h->s.row_bytes;
  return DD_OK;
}

dd_status dd_stream_snapshot(dd_stream h, void* buf, int64_t bytes) {
  if (!h || !buf) return DD_ERR_INVALID_ARG;
  StreamState& s = h->s;
  const int64_t need = 64 + s.tail_rows * s.row_bytes;
  if (bytes < need) return DD_ERR_INVALID_ARG;
  int64_t hdr[8] = {kSnapMagic, s.plan->nchans, s.nbits, s.row_bytes,
                    s.samples_in, s.samples_out, s.tail_rows, s.plan->max_delay};
  std::memcpy(buf, hdr, 64);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && s.tail_rows > 0)
    e = cudaMemcpy(static_cast<uint8_t*>(buf) + 64, s.raw[s.cur].p,
                   (size_t)(s.tail_rows * s.row_bytes), cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

dd_status dd_stream_restore(dd_stream h, const void* buf, int64_t bytes) {
  if (!h || !buf || bytes < 64) return DD_ERR_INVALID_ARG;
  StreamState& s = h->s;
  int64_t hdr[8];
  std::memcpy(hdr, buf, 64);
  if (hdr[0] != kSnapMagic || hdr[1] != s.plan->nchans || hdr[2] != s.nbits ||
      hdr[3] != s.row_bytes || hdr[7] != s.plan->max_delay)
    return DD_ERR_INVALID_ARG;
  const int64_t tail = hdr[6];
  if (tail < 0 || tail > s.cap_rows || bytes < 64 + tail * s.row_bytes) return DD_ERR_INVALID_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && tail > 0)
    e = cudaMemcpy(s.raw[s.cur].p, static_cast<const uint8_t*>(buf) + 64,
                   (size_t)(tail * s.row_bytes), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  s.samples_in = hdr[4];
  s.samples_out = hdr[5];
  s.tail_rows = tail;
  return DD_OK;
}

dd_status dd_batch_create(dd_batch* out) {
  if (!out) return DD_ERR_INVALID_ARG;
  *out = new (std::nothrow) dd_batch_s();
  return *out ? DD_OK : DD_ERR_OOM;
}

void dd_batch_destroy(dd_batch b) { delete b; }

dd_status dd_batch_clear(dd_batch b) {
  if (!b) return DD_ERR_INVALID_ARG;
  b->items.clear();
  return DD_OK;
}

dd_status dd_batch_add(dd_batch b, dd_stream s, const void* in, int64_t n_in, int64_t in_stride,
                       void* out, int64_t out_stride) {
  if (!b || !s || !in || !out || n_in < 0) return DD_ERR_INVALID_ARG;
  if (n_in > s->s.max_gulp || in_stride < s->s.row_bytes || out_stride < n_in ||
      s->s.plan->out_bits != 32)
    return DD_ERR_INVALID_ARG;
  if (!b->items.empty() && b->items[0].stream->s.nbits != s->s.nbits) return DD_ERR_INVALID_ARG;
  for (const BatchItem& it : b->items)
    if (it.stream == s) return DD_ERR_INVALID_ARG;  // one push per stream per batch
  b->items.push_back({s, in, n_in, in_stride, out, out_stride});
  return DD_OK;
}

}  // extern "C"

// All pushes of the batch: per-beam append + corner turn, then the whole
// dedispersion of every beam in one persistent launch (one segment per beam,
// each with its own image, delay table, channel count, trial count and gulp),
// then per-beam tail retention.  `hold` (optional) receives the staging
// tables the launches read (a graph keeps them alive while it exists).
static dd_status batch_launch(dd_batch b, void* cuda_stream, int64_t* nsamps_out,
                              std::vector<std::shared_ptr<StageTab>>* hold) {
  if (!b || !nsamps_out) return DD_ERR_INVALID_ARG;
  if (b->items.empty()) return DD_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nbits = b->items[0].stream->s.nbits;
  int nchans_max = 0;
  for (const BatchItem& it : b->items) nchans_max = std::max(nchans_max, it.stream->s.plan->nchans);
  const int fmt = fmt_for_nbits(nbits, nchans_max);
  const size_t n = b->items.size();
  std::vector<int64_t> totals(n, 0), nouts(n, 0);
  std::vector<DirectJob> jobs;
  std::vector<size_t> job_item;
  for (size_t i = 0; i < n; ++i) {
    BatchItem& it = b->items[i];
    StreamState& s = it.stream->s;
    dd_status r = ensure_device_tables(*s.plan);
    if (r != DD_OK) return r;
    DirectJob job;
    if ((r = stream_stage(s, it.in, it.n_in, it.in_stride, true, st, &job, &nouts[i],
                          &totals[i])) != DD_OK)
      return r;
    if (nouts[i] > 0) {
      job.out = it.out;
      job.out_stride = it.out_stride;
      jobs.push_back(job);
      job_item.push_back(i);
    }
  }
  // Beams run in one persistent launch per tiling: segments carry each
  // beam's tables, and each trial block its own chunk size, so beams of any
  // geometry share a launch (per kMaxSegs beams); beams whose plans were
  // tuned differently (dd_plan_set_tuning, dd_plan_autotune) run in one
  // launch per tiling, each with its own.  Inside a launch, beams of the
  // same shape (channels, trials) are kept adjacent in the work list: on the
  // serving workload, interleaving 512- and 1024-channel beams made the
  // launch 13-26 % slower than the same beams grouped.
  {
    struct Key {
      std::array<int, 3> tile;
      int nchans, ndm;
      size_t job;
    };
    std::vector<Key> key;
    for (size_t k = 0; k < jobs.size(); ++k) {
      const Tuning t = tuning_for(jobs[k].plan->tune, fmt);
      key.push_back({{t.dms_per_block, t.words_per_lane, t.chans_per_chunk}, jobs[k].nchans,
                     jobs[k].ndm, k});
    }
    std::stable_sort(key.begin(), key.end(), [](const Key& a, const Key& b) {
      if (a.tile != b.tile) return a.tile < b.tile;
      if (a.nchans != b.nchans) return a.nchans < b.nchans;
      return a.ndm < b.ndm;
    });
    size_t k0 = 0;
    while (k0 < key.size()) {
      size_t k1 = k0;
      std::vector<DirectJob> part;
      while (k1 < key.size() && part.size() < (size_t)kMaxSegs && key[k1].tile == key[k0].tile)
        part.push_back(jobs[key[k1++].job]);
      // the launch takes the tiling (and status buffer) of its first beam's plan
      Plan& pl = *const_cast<Plan*>(part[0].plan);
      LaunchPlan L;
      std::vector<std::shared_ptr<StageTab>> tabs;
      dd_status r = plan_direct_launch(pl, fmt, fmt == FMT_F32 ? OUT_F32 : OUT_U32,
                                       vmax_for_nbits(nbits), part, &L, &tabs);
      if (r != DD_OK) return r;
      if (hold) hold->insert(hold->end(), tabs.begin(), tabs.end());
      if ((r = run_launch(pl, L, st)) != DD_OK) return r;
      k0 = k1;
    }
  }
  for (size_t i = 0; i < n; ++i) {
    StreamState& s = b->items[i].stream->s;
    dd_status r = keep_tail(s, nouts[i], totals[i], st);
    if (r != DD_OK) return r;
    s.samples_in += b->items[i].n_in;
    s.samples_out += nouts[i];
    nsamps_out[i] = nouts[i];
  }
  return DD_OK;
}

extern "C" {

dd_status dd_batch_launch(dd_batch b, void* cuda_stream, int64_t* nsamps_out) {
  return batch_launch(b, cuda_stream, nsamps_out, nullptr);
}

// Graph capture of a batch launch (steady-state streaming).  The capture
// runs dd_batch_launch's host logic on a capturing stream, so every copy,
// memset and kernel it issues becomes a graph node; the streams' host state
// that the capture advanced is then put back, and each replay advances it.
struct dd_batch_graph_s {
  dd_batch batch = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int cur0 = 0;                   // first stream's tail buffer when variant 0 was taken
  std::vector<int64_t> nouts;     // outputs per add (the same on every replay)
  // staging tables the captured kernels read: held here, so that no later
  // execute, autotune or query on the plans can free them under the graph
  std::vector<std::shared_ptr<StageTab>> tabs;
  ~dd_batch_graph_s() {
    for (auto& e : exec)
      if (e) cudaGraphExecDestroy(e);
  }
};

dd_status dd_batch_graph_create(dd_batch_graph* out, dd_batch b) {
  if (!out || !b || b->items.empty()) return DD_ERR_INVALID_ARG;
  *out = nullptr;
  const size_t n = b->items.size();
  for (const BatchItem& it : b->items) {
    const StreamState& s = it.stream->s;
    if (s.tail_rows != s.plan->max_delay || it.n_in <= 0) return DD_ERR_INVALID_ARG;
  }
  std::unique_ptr<dd_batch_graph_s> g(new (std::nothrow) dd_batch_graph_s());
  if (!g) return DD_ERR_OOM;
  g->batch = b;
  g->nouts.assign(n, 0);
  g->cur0 = b->items[0].stream->s.cur;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_status(e);
  dd_status result = DD_OK;
  for (int v = 0; v < 2 && result == DD_OK; ++v) {
    // save what the capture advances; take variant 1 with the tail buffers swapped
    std::vector<StreamState*> ss;
    std::vector<int> cur;
    std::vector<int64_t> tail, sin, sout;
    std::vector<bool> timing;
    for (BatchItem& it : b->items) {
      StreamState& s = it.stream->s;
      ss.push_back(&s);
      cur.push_back(s.cur);
      tail.push_back(s.tail_rows);
      sin.push_back(s.samples_in);
      sout.push_back(s.samples_out);
      timing.push_back(s.plan->timing);
      s.plan->timing = false;  // no timing events inside a graph
      if (v == 1) s.cur ^= 1;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      result = batch_launch(b, cs, g->nouts.data(), &g->tabs);
      e = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess && result == DD_OK)
        e = cudaGraphInstantiate(&g->exec[v], graph, 0);
      if (graph) cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess && result == DD_OK) result = cuda_status(e);
    for (size_t i = 0; i < ss.size(); ++i) {
      ss[i]->cur = cur[i];
      ss[i]->tail_rows = tail[i];
      ss[i]->samples_in = sin[i];
      ss[i]->samples_out = sout[i];
      ss[i]->plan->timing = timing[i];
    }
  }
  cudaStreamDestroy(cs);
  cudaGetLastError();
  if (result != DD_OK) return result;
  *out = g.release();
  return DD_OK;
}

dd_status dd_batch_graph_launch(dd_batch_graph g, void* cuda_stream, int64_t* nsamps_out) {
  if (!g || !nsamps_out) return DD_ERR_INVALID_ARG;
  dd_batch b = g->batch;
  const int v = b->items[0].stream->s.cur == g->cur0 ? 0 : 1;
  cudaError_t e = cudaGraphLaunch(g->exec[v], static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_status(e);
  for (size_t i = 0; i < b->items.size(); ++i) {
    StreamState& s = b->items[i].stream->s;
    s.samples_in += b->items[i].n_in;
    s.samples_out += g->nouts[i];
    s.cur ^= 1;  // the tail moved to the other buffer
    nsamps_out[i] = g->nouts[i];
  }
  return DD_OK;
}

void dd_batch_graph_destroy(dd_batch_graph g) { delete g; }

// Autotuner: time each compiled tile shape x chunk size on nsamps synthetic
// samples (zeros: the kernel's cost does not depend on the values) and keep
// the fastest.  The paper tuned block shape and samples per thread by hand
// (Sec. 2.3: 8 x 32 on Fermi; Sec. 4.3: 16 x 8 for sub-band).
dd_status dd_plan_autotune(dd_plan plan, int nbits, int64_t nsamps, void* cuda_stream) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || nsamps <= 0) return DD_ERR_INVALID_ARG;
  if (fmt_for_nbits(nbits, p->nchans) < 0) return DD_ERR_UNSUPPORTED_NBITS;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int64_t rb = input_row_bytes(p->nchans, nbits);
  const int64_t rows = nsamps + p->max_delay;
  DevBuf din, dout;
  cudaError_t e = din.ensure((size_t)rows * rb);
  if (e == cudaSuccess) e = dout.ensure((size_t)ndm(*p) * nsamps * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(din.p, 0, din.bytes, st);
  if (e != cudaSuccess) return cuda_status(e);
  cudaEvent_t a = nullptr, z = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaEventCreate(&z)) != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_status(e);
  }
  const Tuning saved = p->tune;
  Tuning best = saved;
  float best_ms = 1e30f;
  static const int ccs[] = {8, 16, 32};
  dd_status result = DD_OK;
  for (int ci = 0; ci < kNumTileCfgs && result == DD_OK; ++ci) {
    for (int cc : ccs) {
      Tuning t;
      t.dms_per_block = kTileCfgs[ci].nwarp * kTileCfgs[ci].dpw;
      t.words_per_lane = kTileCfgs[ci].k;
      t.chans_per_chunk = cc;
      p->tune = t;
      ExecArgs x;
      x.nsamps_out = nsamps;
      x.in = din.p;
      x.in_nbits = nbits;
      x.in_row_stride = rb;
      x.in_rows = rows;
      x.out = dout.p;
      x.out_stride = nsamps;
      x.st = st;
      x.subband = false;
      dd_status r = exec_device(*p, x);  // warm-up (and allocation)
      if (r != DD_OK) continue;          // shape not usable here (e.g. shared memory)
      float ms = 0.f;
      if ((e = cudaEventRecord(a, st)) == cudaSuccess && (r = exec_device(*p, x)) == DD_OK &&
          (e = cudaEventRecord(z, st)) == cudaSuccess && (e = cudaEventSynchronize(z)) == cudaSuccess &&
          (e = cudaEventElapsedTime(&ms, a, z)) == cudaSuccess) {
        if (ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      } else {
        result = r != DD_OK ? r : cuda_status(e);
        break;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  p->tune = (result == DD_OK && best_ms < 1e29f) ? best : saved;
  p->tuned_by_search = result == DD_OK;
  return result;
}

}  // extern "C"
