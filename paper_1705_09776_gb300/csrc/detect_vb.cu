// detect_vb.cu -- K1 launches of variant B: one 512-thread CTA per SM on 128 x 32 tiles, y pass 12 rows per thread.
// The kernel is in detect_kernel.cuh.
#include "detect_kernel.cuh"

namespace cdvs {

cudaError_t launch_detect_b(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, cudaStream_t s) {
  return launch_typed<ShapeB, false>(a, n_tiles, max_radius, storage, n_sms, s);
}

}  // namespace cdvs
