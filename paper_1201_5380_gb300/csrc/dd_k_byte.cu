// Instantiations of the dedispersion kernel for the FMT_BYTE staged format.
#include "dd_dedisp.cuh"

namespace dd {

cudaError_t dispatch_byte(int outk, bool wide, int cfg, bool pbg, const LaunchParams* p, int grid,
                          size_t smem, cudaStream_t st, int* occ) {
  if (outk == OUT_U32)
    return wide ? dispatch_cfg<FMT_BYTE, OUT_U32, true>(cfg, pbg, p, grid, smem, st, occ)
                : dispatch_cfg<FMT_BYTE, OUT_U32, false>(cfg, pbg, p, grid, smem, st, occ);
  if (outk == OUT_HALFIMG && !wide)
    return dispatch_cfg<FMT_BYTE, OUT_HALFIMG, false>(cfg, pbg, p, grid, smem, st, occ);
  if (outk == OUT_NARROW)
    return wide ? dispatch_cfg<FMT_BYTE, OUT_NARROW, true>(cfg, pbg, p, grid, smem, st, occ)
                : dispatch_cfg<FMT_BYTE, OUT_NARROW, false>(cfg, pbg, p, grid, smem, st, occ);
  return cudaErrorInvalidValue;
}

}  // namespace dd
