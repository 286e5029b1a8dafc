// resize.cu -- S0: area-average resize of uneven inputs to a common scale.
//
// The paper brings images to VGA size (larger side 640 px) before
// detection; the resampling method is not stated.  Here output pixel
// (x', y') of a W' x H' image is the mean of the W x H input over
// [x' W / W', (x' + 1) W / W') x [y' H / H', (y' + 1) H / H'], the input
// being constant on each pixel, rounded to the nearest integer (ties to
// even).  Scaled by W' (H'), input column x covers [x W', (x + 1) W') and
// output column x' covers [x' W, (x' + 1) W): every overlap is an integer,
// and the mean is the exact ratio of 64-bit integers
//     sum in[y][x] ox(x', x) oy(y', y) / (W H).
#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

__device__ __forceinline__ long long overlap(int o, int i, int n_in, int n_out) {
  const long long lo = max((long long)o * n_in, (long long)i * n_out);
  const long long hi = min((long long)(o + 1) * n_in, (long long)(i + 1) * n_out);
  return hi > lo ? hi - lo : 0;
}

__global__ void __launch_bounds__(256) resize_kernel(const ResizeJob* jobs) {
  const ResizeJob j = jobs[blockIdx.y];
  const unsigned long long den = (unsigned long long)j.W * j.H;
  const int n = j.W2 * j.H2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int y2 = i / j.W2, x2 = i - (i / j.W2) * j.W2;
    const int y0 = (int)(((long long)y2 * j.H) / j.H2);
    const int y1 = min((int)(((long long)(y2 + 1) * j.H + j.H2 - 1) / j.H2), j.H);
    const int x0 = (int)(((long long)x2 * j.W) / j.W2);
    const int x1 = min((int)(((long long)(x2 + 1) * j.W + j.W2 - 1) / j.W2), j.W);
    unsigned long long s = 0;
    for (int y = y0; y < y1; ++y) {
      const unsigned long long wy = (unsigned long long)overlap(y2, y, j.H, j.H2);
      const uint8_t* row = j.src + (size_t)y * j.pitch;
      unsigned long long sr = 0;
      for (int x = x0; x < x1; ++x) sr += (unsigned long long)row[x] * (unsigned long long)overlap(x2, x, j.W, j.W2);
      s += sr * wy;
    }
    unsigned long long q = s / den;
    const unsigned long long r = s - q * den;
    if (2 * r > den || (2 * r == den && (q & 1ull))) ++q;
    j.dst[(size_t)y2 * j.pitch2 + x2] = (uint8_t)q;
  }
}

}  // namespace

cudaError_t launch_resize(const ResizeJob* d_jobs, int n_jobs, int max_pixels, cudaStream_t s) {
  if (n_jobs <= 0) return cudaSuccess;
  dim3 grid((max_pixels + 255) / 256, n_jobs);
  resize_kernel<<<grid, 256, 0, s>>>(d_jobs);
  return cudaGetLastError();
}

}  // namespace cdvs
