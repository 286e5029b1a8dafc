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

// Overlap of input i with output o in units of 1 / (n_in n_out) of a pixel;
// every product is at most 32768^2 = 2^30, so 32-bit integers hold it.
__device__ __forceinline__ int overlap(int o, int i, int n_in, int n_out) {
  const int lo = max(o * n_in, i * n_out), hi = min((o + 1) * n_in, (i + 1) * n_out);
  return hi > lo ? hi - lo : 0;
}

// Round-to-nearest-even quotient of non-negative integers.
template <typename U>
__device__ __forceinline__ U div_rhe(U num, U den) {
  U q = num / den;
  const U r = num - q * den;
  if (2 * r > den || (2 * r == den && (q & 1))) ++q;
  return q;
}

// One CTA per kRowsPerCta output rows of one image; the row's input rows and
// their weights are shared by its pixels.  Sums and the division run in 32
// bits when 255 W H fits (every image up to 16.8 Mpx), else in 64 bits.
constexpr int kRowsPerCta = 4;

template <typename U>
__device__ __forceinline__ void resize_row(const ResizeJob& j, int y2) {
  const int y0 = (y2 * j.H) / j.H2;
  const int y1 = min(((y2 + 1) * j.H + j.H2 - 1) / j.H2, j.H);
  const U den = (U)j.W * (U)j.H;
  for (int x2 = threadIdx.x; x2 < j.W2; x2 += blockDim.x) {
    const int x0 = (x2 * j.W) / j.W2;
    const int x1 = min(((x2 + 1) * j.W + j.W2 - 1) / j.W2, j.W);
    U s = 0;
    for (int y = y0; y < y1; ++y) {
      const uint8_t* row = j.src + (size_t)y * j.pitch;
      U sr = 0;
      for (int x = x0; x < x1; ++x) sr += (U)row[x] * (U)overlap(x2, x, j.W, j.W2);
      s += sr * (U)overlap(y2, y, j.H, j.H2);
    }
    j.dst[(size_t)y2 * j.pitch2 + x2] = (uint8_t)div_rhe<U>(s, den);
  }
}

__global__ void __launch_bounds__(256) resize_kernel(const ResizeJob* jobs) {
  const ResizeJob j = jobs[blockIdx.y];
  const bool narrow = 255ull * (unsigned long long)j.W * (unsigned long long)j.H < (1ull << 32);
  for (int y2 = blockIdx.x * kRowsPerCta; y2 < min((int)(blockIdx.x + 1) * kRowsPerCta, j.H2); ++y2) {
    if (narrow) resize_row<unsigned>(j, y2);
    else resize_row<unsigned long long>(j, y2);
  }
}

}  // namespace

cudaError_t launch_resize(const ResizeJob* d_jobs, int n_jobs, int max_rows, cudaStream_t s) {
  if (n_jobs <= 0) return cudaSuccess;
  dim3 grid((max_rows + kRowsPerCta - 1) / kRowsPerCta, n_jobs);
  resize_kernel<<<grid, 256, 0, s>>>(d_jobs);
  return cudaGetLastError();
}

}  // namespace cdvs
