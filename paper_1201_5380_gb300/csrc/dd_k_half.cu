// Instantiations of the dedispersion kernel for the FMT_HALF staged format.
#include "dd_dedisp.cuh"

namespace dd {

cudaError_t dispatch_half(int outk, bool wide, int cfg, bool pbg, const LaunchParams* p, int grid,
                          size_t smem, cudaStream_t st, int* occ) {
  if (outk == OUT_U32)
    return wide ? dispatch_cfg<FMT_HALF, OUT_U32, true>(cfg, pbg, p, grid, smem, st, occ)
                : dispatch_cfg<FMT_HALF, OUT_U32, false>(cfg, pbg, p, grid, smem, st, occ);
  if (outk == OUT_HALFIMG && !wide)
    return dispatch_cfg<FMT_HALF, OUT_HALFIMG, false>(cfg, pbg, p, grid, smem, st, occ);
  if (outk == OUT_NARROW)
    return wide ? dispatch_cfg<FMT_HALF, OUT_NARROW, true>(cfg, pbg, p, grid, smem, st, occ)
                : dispatch_cfg<FMT_HALF, OUT_NARROW, false>(cfg, pbg, p, grid, smem, st, occ);
  return cudaErrorInvalidValue;
}

// Multi-tile items: the 16-bit-lane sub-band stages (8-bit input's stage 1,
// every stage 2), tile 5.
cudaError_t dispatch_half_mt(int outk, bool wide, int cfg, bool pbg, const LaunchParams* p,
                             int grid, size_t smem, cudaStream_t st, int* occ) {
  if (cfg != 5) return cudaErrorInvalidValue;
  if (outk == OUT_HALFIMG && !wide)
    return dispatch_mt<FMT_HALF, OUT_HALFIMG, false, 5>(pbg, p, grid, smem, st, occ);
  if (outk == OUT_U32)
    return wide ? dispatch_mt<FMT_HALF, OUT_U32, true, 5>(pbg, p, grid, smem, st, occ)
                : dispatch_mt<FMT_HALF, OUT_U32, false, 5>(pbg, p, grid, smem, st, occ);
  return cudaErrorInvalidValue;
}

}  // namespace dd
