// detect_masked.cu -- K1 launches of the first octave under a block
// proposal (per-tile modes and block masks); the kernel is in
// detect_kernel.cuh.
#include "detect_kernel.cuh"

namespace cdvs {

cudaError_t launch_detect_masked(const DetectArgs& a, int n_tiles, int max_radius, int storage, int grid,
                                 cudaStream_t s) {
  cudaError_t e;
  if (storage == CDVS_STORAGE_FP16) CDVS_LAUNCH_IC(uint8_t, __half, true);
  else CDVS_LAUNCH_IC(uint8_t, float, true);
  return cudaGetLastError();
}

}  // namespace cdvs
