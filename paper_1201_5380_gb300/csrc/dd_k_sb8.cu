// Instantiation of the dedispersion kernel for the FMT_SB8 staged format:
// sub-band stage 2 over an 8-bit-lane stage-1 image (multi-tile items,
// tile 4: 32 trials, 8 words a lane).
#include "dd_dedisp.cuh"

namespace dd {

cudaError_t dispatch_sb8_mt(int outk, bool wide, int cfg, bool pbg, const LaunchParams* p,
                            int grid, size_t smem, cudaStream_t st, int* occ) {
  if (outk == OUT_U32 && !wide && cfg == 4)
    return dispatch_mt<FMT_SB8, OUT_U32, false, 4>(pbg, p, grid, smem, st, occ);
  return cudaErrorInvalidValue;
}

}  // namespace dd
