// Instantiations of the dedispersion kernel for the FMT_NIB staged format.
#include "dd_dedisp.cuh"

namespace dd {

cudaError_t dispatch_nib(int outk, bool wide, int cfg, bool pbg, const LaunchParams* p, int grid,
                          size_t smem, cudaStream_t st, int* occ) {
  if (outk == OUT_U32)
    return wide ? dispatch_cfg<FMT_NIB, OUT_U32, true>(cfg, pbg, p, grid, smem, st, occ)
                : dispatch_cfg<FMT_NIB, OUT_U32, false>(cfg, pbg, p, grid, smem, st, occ);
  if (outk == OUT_HALFIMG && !wide)
    return dispatch_cfg<FMT_NIB, OUT_HALFIMG, false>(cfg, pbg, p, grid, smem, st, occ);
  if (outk == OUT_NARROW)
    return wide ? dispatch_cfg<FMT_NIB, OUT_NARROW, true>(cfg, pbg, p, grid, smem, st, occ)
                : dispatch_cfg<FMT_NIB, OUT_NARROW, false>(cfg, pbg, p, grid, smem, st, occ);
  return cudaErrorInvalidValue;
}

// Multi-tile items: 1- and 2-bit sub-band stage 1 (16- or 8-bit image
// output), tile 0.  The 8-bit image is written by this kernel only.
cudaError_t dispatch_nib_mt(int outk, bool wide, int cfg, bool pbg, const LaunchParams* p,
                            int grid, size_t smem, cudaStream_t st, int* occ) {
  if (outk == OUT_HALFIMG && !wide && cfg == 0)
    return dispatch_mt<FMT_NIB, OUT_HALFIMG, false, 0>(pbg, p, grid, smem, st, occ);
  if (outk == OUT_BYTEIMG && !wide && cfg == 0)
    return dispatch_mt<FMT_NIB, OUT_BYTEIMG, false, 0>(pbg, p, grid, smem, st, occ);
  return cudaErrorInvalidValue;
}

}  // namespace dd
