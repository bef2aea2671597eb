// Instantiations of the dedispersion kernel for the 32-bit staged formats
// (unsigned sums of sub-band stage 2 with wide intermediates, and float).
#include "dd_dedisp.cuh"

namespace dd {

cudaError_t dispatch_word(int fmt, int outk, bool wide, int cfg, bool pbg, const LaunchParams* p,
                          int grid, size_t smem, cudaStream_t st, int* occ) {
  (void)wide;
  if (fmt == FMT_U32 && outk == OUT_U32)
    return dispatch_cfg<FMT_U32, OUT_U32, false>(cfg, pbg, p, grid, smem, st, occ);
  if (fmt == FMT_U32 && outk == OUT_NARROW)
    return dispatch_cfg<FMT_U32, OUT_NARROW, false>(cfg, pbg, p, grid, smem, st, occ);
  if (fmt == FMT_F32 && outk == OUT_F32)
    return dispatch_cfg<FMT_F32, OUT_F32, false>(cfg, pbg, p, grid, smem, st, occ);
  return cudaErrorInvalidValue;
}

}  // namespace dd
