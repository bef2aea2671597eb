// Instantiations of the dedispersion kernel for the FMT_TRI staged format
// (8-bit input, three samples a word in 10-bit lanes; 32-bit sums always).
#include "dd_dedisp.cuh"

namespace dd {

cudaError_t dispatch_tri(int outk, bool /*wide*/, int cfg, bool pbg, const LaunchParams* p,
                         int grid, size_t smem, cudaStream_t st, int* occ) {
  if (outk == OUT_U32) return dispatch_cfg<FMT_TRI, OUT_U32, false>(cfg, pbg, p, grid, smem, st, occ);
  if (outk == OUT_NARROW)
    return dispatch_cfg<FMT_TRI, OUT_NARROW, false>(cfg, pbg, p, grid, smem, st, occ);
  return cudaErrorInvalidValue;
}

}  // namespace dd
