// detect_vc.cu -- K1 launches of variant C: two 256-thread CTAs per SM on 128 x 16 tiles, y pass 4 rows per thread.
// The kernel is in detect_kernel.cuh.
#include "detect_kernel.cuh"

namespace cdvs {

cudaError_t launch_detect_c(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, cudaStream_t s) {
  return launch_typed<ShapeC, false>(a, n_tiles, max_radius, storage, n_sms, s);
}

}  // namespace cdvs
