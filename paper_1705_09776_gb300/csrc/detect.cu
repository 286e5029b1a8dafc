// detect.cu -- K1 launches of the plain detector (the kernel is in
// detect_kernel.cuh; the variants under a block proposal are instantiated in
// detect_masked.cu, so the two compile in parallel).
#include "detect_kernel.cuh"

namespace cdvs {

size_t detect_smem_bytes(int max_radius) { return detect_smem(max_radius, 4, 0); }

cudaError_t launch_detect(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms,
                          cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  if (max_radius > kMaxRadius) return cudaErrorInvalidValue;
  const int grid = n_tiles < n_sms ? n_tiles : n_sms;
  cudaError_t e;
  const bool masked = a.tile_mode && a.block_mask;
  if (masked && a.octave != 0) return cudaErrorInvalidValue;  // proposals mask the first octave only
  if (masked) return launch_detect_masked(a, n_tiles, max_radius, storage, grid, s);
  if (storage == CDVS_STORAGE_FP16) {
    if (a.octave == 0) CDVS_LAUNCH_IC(uint8_t, __half, false);
    else CDVS_LAUNCH_IC(__half, __half, false);
  } else {
    if (a.octave == 0) CDVS_LAUNCH_IC(uint8_t, float, false);
    else CDVS_LAUNCH_IC(float, float, false);
  }
  return cudaGetLastError();
}

}  // namespace cdvs
