// Serving engine: gulps of many beams as they arrive, continuously batched.
//
// Each beam is a stream (device-resident overlap tail, dd_stream_*); the
// engine queues submitted gulps, admits them into launches as in-flight
// launches retire and arena space frees up, and runs each launch as
//   inputs host -> arena          (copy stream `h2d`)
//   one dd_batch_launch           (compute stream, waits for the inputs)
//   outputs arena -> host         (copy stream `d2h`, waits for the compute)
// so the input copies of launch k+1 and the output copies of launch k-1
// overlap the compute of launch k.  Completion times are stamped by host
// functions queued behind the work, so latency is submit -> output ready.
// The paper has no serving layer; this is the runtime around its transform.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <vector>

#include "dd_internal.h"

namespace dd {
namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr size_t kGranule = 256;
size_t round_up(size_t n) { return (n + kGranule - 1) & ~(kGranule - 1); }

// First-fit allocator over one device allocation; frees coalesce with their
// neighbours.  Offsets and sizes are multiples of 256 bytes.
class Arena {
 public:
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  cudaError_t init(size_t bytes) {
    total_ = bytes & ~(kGranule - 1);
    if (total_ == 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&base_), total_);
    if (e != cudaSuccess) {
      base_ = nullptr;
      return e;
    }
    free_[0] = total_;
    return cudaSuccess;
  }
  bool alloc(size_t n, size_t* off) {
    n = round_up(std::max<size_t>(n, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n;
      const size_t at = it->first + n;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += n;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = round_up(std::max<size_t>(n, 1));
    used_ -= n;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }
  bool fits_ever(size_t n) const { return round_up(std::max<size_t>(n, 1)) <= total_; }
  uint8_t* base() const { return base_; }
  size_t used() const { return used_; }

 private:
  uint8_t* base_ = nullptr;
  size_t total_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes
};

struct Beam {
  dd_plan plan;
  dd_stream stream;
  int nbits;
  int64_t max_gulp;
  int64_t row_bytes;
  int ndm;
};

struct Request {
  uint64_t id = 0;
  int beam = 0;
  const void* in = nullptr;
  int64_t n_in = 0, in_stride = 0;
  void* host_out = nullptr;
  int64_t host_stride = 0;
  int64_t t_submit = 0;
  size_t in_off = 0, in_bytes = 0, out_off = 0, out_bytes = 0;
  bool has_in_buf = false, has_out_buf = false;
  int64_t dev_stride = 0;
  int64_t n_out = 0;
  int status = DD_OK;
  double latency_ms = 0.0;
};

struct Launch {
  std::vector<uint64_t> reqs;
  double pause_ms = 0.0;                // host-side pause queued before the transform
  cudaEvent_t done = nullptr;           // after everything of the launch
  std::atomic<int64_t> t_compute{0};    // stamped behind the transform
  std::atomic<int64_t> t_copied{0};     // stamped behind the output copies
};

void CUDART_CB stamp(void* slot) {
  static_cast<std::atomic<int64_t>*>(slot)->store(now_ns());
}

// A pause of the compute stream on the host (dd_server_pause_next_launch):
// the stream waits for this callback; no device work is involved.
void CUDART_CB pause_host(void* ms) {
  std::this_thread::sleep_for(
      std::chrono::microseconds((int64_t)(*static_cast<double*>(ms) * 1000.0)));
}

// Wait for an event, at most timeout_ms (<= 0: no limit).  The wait polls,
// so a GPU that stops answering turns into DD_ERR_TIMEOUT on the host.
dd_status wait_event(cudaEvent_t ev, double timeout_ms) {
  if (timeout_ms <= 0.0) return cuda_status(cudaEventSynchronize(ev));
  const int64_t deadline = now_ns() + (int64_t)(timeout_ms * 1e6);
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return DD_OK;
    if (e != cudaErrorNotReady) return cuda_status(e);
    if (now_ns() >= deadline) return DD_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int64_t input_row_bytes(int nchans, int nbits) {
  return nbits == 32 ? (int64_t)nchans * 4 : ((int64_t)nchans * nbits + 7) / 8;
}

}  // namespace
}  // namespace dd

using namespace dd;

struct dd_server_s {
  std::mutex mu;
  int device = 0;
  Arena arena;
  int max_batch = 1, max_inflight = 1;
  cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
  dd_batch batch = nullptr;
  std::vector<Beam> beams;
  std::map<uint64_t, Request> reqs;
  std::deque<uint64_t> queue;                   // submitted, not admitted
  std::deque<std::unique_ptr<Launch>> inflight;  // launch order
  std::deque<uint64_t> completed;               // not yet polled
  uint64_t next_id = 1;
  double timeout_ms = 0.0;    // deadline of host waits (<= 0: none)
  double pause_next_ms = 0.0; // dd_server_pause_next_launch

  ~dd_server_s() {
    for (auto& l : inflight)
      if (l->done) {
        cudaEventSynchronize(l->done);
        cudaEventDestroy(l->done);
      }
    for (Beam& b : beams) dd_stream_destroy(b.stream);
    if (batch) dd_batch_destroy(batch);
    if (h2d) cudaStreamDestroy(h2d);
    if (comp) cudaStreamDestroy(comp);
    if (d2h) cudaStreamDestroy(d2h);
  }

  void free_request_buffers(Request& r, bool keep_out) {
    if (r.has_in_buf) arena.release(r.in_off, r.in_bytes);
    r.has_in_buf = false;
    if (r.has_out_buf && !keep_out) {
      arena.release(r.out_off, r.out_bytes);
      r.has_out_buf = false;
    }
  }

  // Retire launches whose work has finished (in launch order).  With
  // wait_front, first wait for the oldest launch (at most timeout_ms); a
  // launch still running at the deadline stays in flight and DD_ERR_TIMEOUT
  // is returned.
  dd_status retire(bool wait_front) {
    while (!inflight.empty()) {
      Launch& l = *inflight.front();
      if (wait_front) {
        const dd_status w = wait_event(l.done, timeout_ms);
        if (w != DD_OK) return w;
        wait_front = false;
      } else if (cudaEventQuery(l.done) != cudaSuccess) {
        break;
      }
      for (uint64_t id : l.reqs) {
        Request& r = reqs[id];
        const int64_t t = r.host_out ? l.t_copied.load() : l.t_compute.load();
        r.latency_ms = (double)(t - r.t_submit) / 1e6;
        free_request_buffers(r, r.host_out == nullptr && r.status == DD_OK);
        completed.push_back(id);
      }
      cudaEventDestroy(l.done);
      inflight.pop_front();
    }
    return DD_OK;
  }

  // Fail a launch that could not be issued: its requests complete with `st`.
  void fail(std::vector<uint64_t>& ids, dd_status st) {
    for (uint64_t id : ids) {
      Request& r = reqs[id];
      r.status = st;
      free_request_buffers(r, false);
      completed.push_back(id);
    }
  }

  // Admit queued gulps into one launch and issue it; returns the count.
  int admit_and_launch(dd_status* err) {
    *err = DD_OK;
    if ((int)inflight.size() >= max_inflight || queue.empty()) return 0;
    std::vector<uint64_t> take;
    std::set<int> in_launch, blocked;
    int nbits = -1;
    for (uint64_t id : queue) {
      if ((int)take.size() >= max_batch) break;
      Request& r = reqs[id];
      if (in_launch.count(r.beam) || blocked.count(r.beam)) {
        blocked.insert(r.beam);  // keep the beam's order
        continue;
      }
      const Beam& b = beams[r.beam];
      if (nbits >= 0 && b.nbits != nbits) {
        blocked.insert(r.beam);
        continue;
      }
      r.dev_stride = (r.n_in + 3) & ~(int64_t)3;
      r.in_bytes = (size_t)(r.n_in * b.row_bytes);
      r.out_bytes = (size_t)b.ndm * (size_t)r.dev_stride * 4u;
      size_t a = 0, o = 0;
      if (!arena.alloc(r.in_bytes, &a)) {
        blocked.insert(r.beam);
        continue;
      }
      if (!arena.alloc(r.out_bytes, &o)) {
        arena.release(a, r.in_bytes);
        blocked.insert(r.beam);
        continue;
      }
      r.in_off = a;
      r.out_off = o;
      r.has_in_buf = r.has_out_buf = true;
      nbits = b.nbits;
      in_launch.insert(r.beam);
      take.push_back(id);
    }
    if (take.empty()) return 0;
    std::set<uint64_t> taken(take.begin(), take.end());
    queue.erase(std::remove_if(queue.begin(), queue.end(),
                               [&](uint64_t id) { return taken.count(id) != 0; }),
                queue.end());

    std::unique_ptr<Launch> L(new Launch);
    L->reqs = take;
    uint8_t* base = arena.base();
    cudaError_t e = cudaSuccess;
    // inputs in
    for (uint64_t id : take) {
      Request& r = reqs[id];
      const Beam& b = beams[r.beam];
      if (r.n_in > 0 && e == cudaSuccess)
        e = cudaMemcpy2DAsync(base + r.in_off, b.row_bytes, r.in, r.in_stride, b.row_bytes,
                              r.n_in, cudaMemcpyHostToDevice, h2d);
    }
    cudaEvent_t ev_in = nullptr, ev_comp = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(comp, ev_in, 0);
    if (ev_in) cudaEventDestroy(ev_in);
    if (e != cudaSuccess) {
      *err = cuda_status(e);
      fail(take, *err);
      return 0;
    }
    // one batched launch over every admitted beam
    dd_batch_clear(batch);
    dd_status s = DD_OK;
    for (uint64_t id : take) {
      Request& r = reqs[id];
      const Beam& b = beams[r.beam];
      if (s == DD_OK)
        s = dd_batch_add(batch, b.stream, base + r.in_off, r.n_in, b.row_bytes, base + r.out_off,
                         r.dev_stride);
    }
    std::vector<int64_t> nouts(take.size(), 0);
    if (s == DD_OK) s = dd_batch_launch(batch, comp, nouts.data());
    if (s != DD_OK) {
      *err = s;
      fail(take, s);
      return 0;
    }
    bool any_host = false;
    for (size_t i = 0; i < take.size(); ++i) {
      Request& r = reqs[take[i]];
      r.n_out = nouts[i];
      any_host = any_host || r.host_out != nullptr;
    }
    // a requested pause holds the launch back after its transform is queued
    // (so that none of the launch's own set-up waits for it)
    if (pause_next_ms > 0.0) {
      L->pause_ms = pause_next_ms;
      pause_next_ms = 0.0;
      e = cudaLaunchHostFunc(comp, pause_host, &L->pause_ms);
    }
    if (e == cudaSuccess) e = cudaLaunchHostFunc(comp, stamp, &L->t_compute);
    cudaStream_t last = comp;
    if (e == cudaSuccess && any_host) {
      e = cudaEventCreateWithFlags(&ev_comp, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(ev_comp, comp);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(d2h, ev_comp, 0);
      if (ev_comp) cudaEventDestroy(ev_comp);
      for (uint64_t id : take) {
        Request& r = reqs[id];
        if (!r.host_out || r.n_out == 0 || e != cudaSuccess) continue;
        e = cudaMemcpy2DAsync(r.host_out, (size_t)r.host_stride * 4, base + r.out_off,
                              (size_t)r.dev_stride * 4, (size_t)r.n_out * 4, beams[r.beam].ndm,
                              cudaMemcpyDeviceToHost, d2h);
      }
      if (e == cudaSuccess) e = cudaLaunchHostFunc(d2h, stamp, &L->t_copied);
      last = d2h;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(L->done, last);
    if (e != cudaSuccess) {
      // the transform is queued: wait for it before handing buffers back
      cudaStreamSynchronize(comp);
      cudaStreamSynchronize(d2h);
      if (L->done) cudaEventDestroy(L->done);
      *err = cuda_status(e);
      fail(take, *err);
      return 0;
    }
    inflight.push_back(std::move(L));
    return (int)take.size();
  }
};

extern "C" {

dd_status dd_server_create(dd_server* out, size_t arena_bytes, int max_batch, int max_inflight) {
  if (!out) return DD_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_batch < 1 || max_batch > kMaxSegs || max_inflight < 1 || max_inflight > 8 ||
      arena_bytes < kGranule)
    return DD_ERR_INVALID_ARG;
  std::unique_ptr<dd_server_s> s(new (std::nothrow) dd_server_s());
  if (!s) return DD_ERR_OOM;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) return cuda_status(e);
  s->max_batch = max_batch;
  s->max_inflight = max_inflight;
  if ((e = cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->comp, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_status(e);
  if ((e = s->arena.init(arena_bytes)) != cudaSuccess)
    return e == cudaErrorMemoryAllocation ? DD_ERR_OOM : cuda_status(e);
  dd_status st = dd_batch_create(&s->batch);
  if (st != DD_OK) return st;
  *out = s.release();
  return DD_OK;
}

void dd_server_destroy(dd_server s) {
  if (!s) return;
  cudaSetDevice(s->device);
  delete s;
}

dd_status dd_server_add_beam(dd_server s, dd_plan plan, int nbits, int64_t max_gulp, int* beam) {
  if (!s || !plan || !beam || max_gulp <= 0) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  cudaSetDevice(s->device);
  int32_t nch = 0, ndm = 0;
  dd_status st = dd_plan_get_dm_count(plan, &ndm);
  if (st != DD_OK) return st;
  Plan* p = reinterpret_cast<Plan*>(plan);
  nch = p->nchans;
  dd_stream stream = nullptr;
  if ((st = dd_stream_create(&stream, plan, nbits, max_gulp)) != DD_OK) return st;
  s->beams.push_back({plan, stream, nbits, max_gulp, input_row_bytes(nch, nbits), (int)ndm});
  *beam = (int)s->beams.size() - 1;
  return DD_OK;
}

dd_status dd_server_submit(dd_server s, int beam, const void* in, int64_t n_in,
                           int64_t in_stride, void* host_out, int64_t out_stride,
                           uint64_t* request) {
  if (!s || !in || !request || n_in < 0) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (beam < 0 || beam >= (int)s->beams.size()) return DD_ERR_INVALID_ARG;
  const Beam& b = s->beams[beam];
  if (n_in > b.max_gulp || in_stride < b.row_bytes) return DD_ERR_INVALID_ARG;
  if (host_out && out_stride < n_in) return DD_ERR_INVALID_ARG;
  const int64_t stride = (n_in + 3) & ~(int64_t)3;
  if (!s->arena.fits_ever(round_up((size_t)(n_in * b.row_bytes) + 1) +
                          (size_t)b.ndm * (size_t)stride * 4u))
    return DD_ERR_REJECTED;
  Request r;
  r.id = s->next_id++;
  r.beam = beam;
  r.in = in;
  r.n_in = n_in;
  r.in_stride = in_stride;
  r.host_out = host_out;
  r.host_stride = out_stride;
  r.t_submit = now_ns();
  s->reqs[r.id] = r;
  s->queue.push_back(r.id);
  *request = r.id;
  return DD_OK;
}

dd_status dd_server_step(dd_server s, int wait, int* admitted) {
  if (!s) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  cudaSetDevice(s->device);
  s->retire(false);
  dd_status err = DD_OK;
  int n = s->admit_and_launch(&err);
  if (n == 0 && err == DD_OK && wait && !s->inflight.empty()) {
    err = s->retire(true);
    if (err == DD_OK) n = s->admit_and_launch(&err);
  }
  if (admitted) *admitted = n;
  return err;
}

dd_status dd_server_set_timeout(dd_server s, double timeout_ms) {
  if (!s || !(timeout_ms >= 0.0)) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->timeout_ms = timeout_ms;
  return DD_OK;
}

dd_status dd_server_drain(dd_server s) {
  if (!s) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  cudaSetDevice(s->device);
  const int64_t deadline = now_ns() + (int64_t)(s->timeout_ms * 1e6);
  while (!s->inflight.empty()) {
    const double left = s->timeout_ms > 0.0 ? (double)(deadline - now_ns()) / 1e6 : 0.0;
    if (s->timeout_ms > 0.0 && left <= 0.0) return DD_ERR_TIMEOUT;
    const dd_status w = wait_event(s->inflight.front()->done, left);
    if (w != DD_OK) return w;
    s->retire(false);
  }
  return DD_OK;
}

dd_status dd_server_pause_next_launch(dd_server s, double ms) {
  if (!s || !(ms >= 0.0) || ms > 60000.0) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->pause_next_ms = ms;
  return DD_OK;
}

dd_status dd_server_poll(dd_server s, dd_request_info* out, int max, int* n) {
  if (!s || !n || (max > 0 && !out)) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  cudaSetDevice(s->device);
  s->retire(false);
  int k = 0;
  while (k < max && !s->completed.empty()) {
    const uint64_t id = s->completed.front();
    s->completed.pop_front();
    Request& r = s->reqs[id];
    dd_request_info& o = out[k++];
    o.request = id;
    o.beam = r.beam;
    o.status = r.status;
    o.nsamps_out = r.n_out;
    o.out_dev = r.has_out_buf ? s->arena.base() + r.out_off : nullptr;
    o.out_stride = r.dev_stride;
    o.latency_ms = r.latency_ms;
    if (!r.has_out_buf) s->reqs.erase(id);
  }
  *n = k;
  return DD_OK;
}

dd_status dd_server_copy_out(dd_server s, uint64_t request, void* host_dst, int64_t host_stride) {
  if (!s || !host_dst) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request);
  if (it == s->reqs.end() || !it->second.has_out_buf) return DD_ERR_INVALID_ARG;
  Request& r = it->second;
  if (std::find(s->queue.begin(), s->queue.end(), request) != s->queue.end())
    return DD_ERR_NOT_READY;
  for (auto& l : s->inflight)
    if (std::find(l->reqs.begin(), l->reqs.end(), request) != l->reqs.end())
      return DD_ERR_NOT_READY;
  if (host_stride < r.n_out) return DD_ERR_INVALID_ARG;
  if (r.n_out == 0) return DD_OK;
  cudaSetDevice(s->device);
  cudaError_t e = cudaMemcpy2D(host_dst, (size_t)host_stride * 4, s->arena.base() + r.out_off,
                               (size_t)r.dev_stride * 4, (size_t)r.n_out * 4,
                               s->beams[r.beam].ndm, cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

dd_status dd_server_release(dd_server s, uint64_t request) {
  if (!s) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request);
  if (it == s->reqs.end() || !it->second.has_out_buf) return DD_ERR_INVALID_ARG;
  if (std::find(s->queue.begin(), s->queue.end(), request) != s->queue.end())
    return DD_ERR_NOT_READY;
  for (auto& l : s->inflight)
    if (std::find(l->reqs.begin(), l->reqs.end(), request) != l->reqs.end())
      return DD_ERR_NOT_READY;
  if (std::find(s->completed.begin(), s->completed.end(), request) != s->completed.end())
    return DD_ERR_NOT_READY;  // poll it first
  s->free_request_buffers(it->second, false);
  s->reqs.erase(it);
  return DD_OK;
}

dd_status dd_server_stats(dd_server s, int* queued, int* inflight, int* completed,
                          size_t* arena_used) {
  if (!s) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int inf = 0;
  for (auto& l : s->inflight) inf += (int)l->reqs.size();
  if (queued) *queued = (int)s->queue.size();
  if (inflight) *inflight = inf;
  if (completed) *completed = (int)s->reqs.size() - (int)s->queue.size() - inf;
  if (arena_used) *arena_used = s->arena.used();
  return DD_OK;
}

}  // extern "C"
