// dd_execute_noalloc: the direct transform for callers that may not allocate
// device memory.  Everything the kernels need besides the caller's input and
// output (staged image, trial-block and staging tables, kill mask, status
// word) lives in one fixed file-scope device array, so no call allocates or
// frees.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "dd_internal.h"

namespace dd {
namespace {

static_assert(DD_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");

// The shared scratch.  Every GPU that loads the library holds it until the
// process exits.  In host code this name is only a host-side stand-in: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).
dd_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= kMaxDevices) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e);
    g_scratch_ptr[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return DD_OK;
}

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" dd_status dd_execute_noalloc(dd_plan plan, int64_t nsamps_out, const void* in,
                                        int in_nbits, int64_t in_row_stride, void* out,
                                        int64_t out_stride, void* cuda_stream) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !in || !out || nsamps_out <= 0 || out_stride < nsamps_out) return DD_ERR_INVALID_ARG;
  const int fmt = fmt_for_nbits(in_nbits, p->nchans);
  if (fmt < 0) return DD_ERR_UNSUPPORTED_NBITS;
  if (p->dms.empty()) return DD_ERR_NO_DM_LIST;
  if (p->out_bits != 32) return DD_ERR_INVALID_ARG;
  const int64_t row_bytes =
      in_nbits == 32 ? (int64_t)p->nchans * 4 : ((int64_t)p->nchans * in_nbits + 7) / 8;
  if (in_row_stride < row_bytes) return DD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(p->mu);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* sc = nullptr;
  dd_status s = scratch_for_current_device(&sc);
  if (s != DD_OK) return s;

  // Plan the launch first, with the staging tables left on the host: they
  // size the scratch.  Device pointers are patched in once it is laid out.
  const int cfg = tile_cfg_index(tuning_for(p->tune, fmt));
  const int B = kTileCfgs[cfg].nwarp * kTileCfgs[cfg].dpw;
  const int bi = b_index(B);
  const std::vector<int32_t>& blocks = p->blocks_B[bi];
  const int64_t rw = image_row_words(fmt, tuning_for(p->tune, fmt), nsamps_out, p->max_delay, p->spread_B[bi]);
  DirectJob j;
  j.img = reinterpret_cast<const uint32_t*>(sc);
  j.row_words = rw;
  j.img_row_samples = rw * fmt_spw(fmt);
  j.d_delays = nullptr;
  j.h_delays = p->delays.data();
  j.nchans = p->nchans;
  j.ndm = ndm(*p);
  j.nsamps = nsamps_out;
  j.out = out;
  j.out_stride = out_stride;
  j.plan = p;
  j.blk_dev = reinterpret_cast<const int32_t*>(sc);
  j.no_upload = true;
  LaunchPlan L;
  std::vector<std::shared_ptr<StageTab>> tabs;
  s = plan_direct_launch(*p, fmt, fmt == FMT_F32 ? OUT_F32 : OUT_U32, vmax_for_nbits(in_nbits),
                         {j}, &L, &tabs);
  if (s != DD_OK) return s;
  if (L.lp.n_items == 0)  // nothing to launch: only the status word is reset
    return cuda_status(cudaMemsetAsync(sc, 0, 16, st));
  const std::shared_ptr<StageTab> t = tabs.at(0);

  // Layout of the scratch for this call; reject problems that do not fit.
  const size_t off_status = 0;
  const size_t off_mask = 256;
  const size_t off_blocks = off_mask + round256((size_t)p->nchans);
  const size_t off_atab = off_blocks + round256(blocks.size() * sizeof(int32_t));
  const size_t off_crec = off_atab + round256(t->atab.size() * sizeof(uint32_t));
  const size_t off_image = off_crec + round256(t->crec.size() * sizeof(int32_t));
  const size_t need = off_image + (size_t)p->nchans * (size_t)rw * 4u;
  if (need > (size_t)DD_NOALLOC_SCRATCH_BYTES) return DD_ERR_OOM;
  uint32_t* status = reinterpret_cast<uint32_t*>(sc + off_status);
  uint8_t* mask = sc + off_mask;
  int32_t* blk = reinterpret_cast<int32_t*>(sc + off_blocks);
  uint32_t* atab = reinterpret_cast<uint32_t*>(sc + off_atab);
  int32_t* crec = reinterpret_cast<int32_t*>(sc + off_crec);
  uint32_t* img = reinterpret_cast<uint32_t*>(sc + off_image);

  // The array keeps the previous call's contents: reset the status word and
  // reload the tables (the image is fully rewritten by the corner turn).
  cudaError_t e = cudaMemsetAsync(status, 0, 16, st);  // status word and item counter
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mask, p->mask.data(), (size_t)p->nchans, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(blk, blocks.data(), blocks.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(atab, t->atab.data(), t->atab.size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(crec, t->crec.data(), t->crec.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);

  const int64_t rows = nsamps_out + p->max_delay;
  e = launch_corner_turn(in_nbits, fmt, static_cast<const uint8_t*>(in), in_row_stride, 0, rows,
                         p->nchans, mask, img, rw, 0, rw, st);
  if (e != cudaSuccess) return cuda_status(e);

  Seg& g = L.lp.segs[0];
  g.img = img;
  g.blk = blk;
  g.atab = atab;
  g.crec = crec;
  L.lp.status = status;
  L.lp.next_item = reinterpret_cast<unsigned long long*>(sc + off_status + 8);
  return cuda_status(launch_dedisp(L.fmt, L.outk, L.wide, L.cfg, L.lp, L.grid, L.smem, st));
}

extern "C" dd_status dd_noalloc_get_device_status(void* cuda_stream, uint32_t* flags) {
  if (!flags) return DD_ERR_INVALID_ARG;
  *flags = 0;
  unsigned char* sc = nullptr;
  dd_status s = scratch_for_current_device(&sc);
  if (s != DD_OK) return s;
  // The status word sits at the start of the scratch; each dd_execute_noalloc
  // call resets it on its stream before its kernels run.
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, sc, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  *flags = v;
  return DD_OK;
}
