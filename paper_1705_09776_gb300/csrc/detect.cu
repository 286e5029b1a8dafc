// detect.cu -- K1 launches of the plain detector, variant A (one 512-thread
// CTA per SM on 128 x 32 tiles, y pass 6 rows per thread), and the dispatch
// over the variants.  The kernel is in detect_kernel.cuh; every variant is
// instantiated in a translation unit of its own (detect_v*.cu, and
// detect_masked.cu for the variants under a block proposal), so they compile
// in parallel.
#include "detect_kernel.cuh"

namespace cdvs {

size_t detect_smem_bytes(int max_radius) { return detect_smem<ShapeA>(max_radius, 4, 0); }

int detect_variant_rows(int variant) {
  switch (variant) {
    case 1: return ShapeB::TY;
    case 2: return ShapeC::TY;
    case 3: return ShapeD::TY;
    default: return ShapeA::TY;
  }
}

const char* detect_variant_name(int variant) {
  switch (variant) {
    case 1: return "128x32 tile, 512 threads x 1 CTA/SM, y pass 12 rows/thread";
    case 2: return "128x16 tile, 256 threads x 2 CTAs/SM, y pass 4 rows/thread";
    case 3: return "128x16 tile, 256 threads x 2 CTAs/SM, y pass 10 rows/thread";
    default: return "128x32 tile, 512 threads x 1 CTA/SM, y pass 6 rows/thread";
  }
}

cudaError_t launch_detect_a(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, cudaStream_t s) {
  return launch_typed<ShapeA, false>(a, n_tiles, max_radius, storage, n_sms, s);
}

cudaError_t launch_detect(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, int variant,
                          cudaStream_t s) {
  // n_tiles = 0 launches nothing but loads the variant's kernel and sets its
  // shared-memory attribute (the tuner does this before timing a variant)
  if (n_tiles < 0) return cudaSuccess;
  if (max_radius > kMaxRadius) return cudaErrorInvalidValue;
  const bool masked = a.tile_mode && a.block_mask;
  if (masked && (a.octave != 0 || variant != 0)) return cudaErrorInvalidValue;  // first octave, 128 x 32 tiles
  if (masked) return launch_detect_masked(a, n_tiles, max_radius, storage, n_sms, s);
  switch (variant) {
    case 0: return launch_detect_a(a, n_tiles, max_radius, storage, n_sms, s);
    case 1: return launch_detect_b(a, n_tiles, max_radius, storage, n_sms, s);
    case 2: return launch_detect_c(a, n_tiles, max_radius, storage, n_sms, s);
    case 3: return launch_detect_d(a, n_tiles, max_radius, storage, n_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cdvs
