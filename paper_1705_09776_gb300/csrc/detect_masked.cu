// detect_masked.cu -- K1 launches of the first octave under a block
// proposal (per-tile modes and block masks), on variant A's 128 x 32 tiles;
// the kernel is in detect_kernel.cuh.
#include "detect_kernel.cuh"

namespace cdvs {

cudaError_t launch_detect_masked(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms,
                                 cudaStream_t s) {
  return launch_typed<ShapeA, true>(a, n_tiles, max_radius, storage, n_sms, s);
}

}  // namespace cdvs
