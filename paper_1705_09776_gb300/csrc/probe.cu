// probe.cu -- the measured rate of packed FP32 multiply-adds (fma.rn.f32x2)
// on the context's GPU: the rate K1's filters and fit run at, reported beside
// the peak derived from the SM count, 128 FP32 lanes per SM and the maximum
// clock.  A register-only loop: every thread advances eight independent
// chains of packed FMAs, and the grid fills every SM with 2048 threads.
#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kProbeThreads = 256, kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) ffma2_rate_kernel(float* out, int iters, float seed) {
  float2 x[kProbeChains];
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) x[q] = make_float2(seed + (float)q, seed - (float)q);
  const float2 m = make_float2(0.999f, 0.999f), c = make_float2(1.0e-3f, 1.0e-3f);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) x[q] = __ffma2_rn(x[q], m, c);
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) s += x[q].x + x[q].y;
  if (s == -1.0f) out[threadIdx.x] = s;  // never true for a positive seed; keeps the chains live
}

}  // namespace

cudaError_t probe_ffma2(int n_sms, double* tflops) {
  *tflops = 0.0;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float* out = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * kProbeThreads);
  const int grid = n_sms * (2048 / kProbeThreads), iters = 1 << 16;
  float ms = 0.0f;
  if (e == cudaSuccess) {
    ffma2_rate_kernel<<<grid, kProbeThreads, 0, s>>>(out, iters / 16, 1.0f);  // warm-up
    cudaEventRecord(e0, s);
    ffma2_rate_kernel<<<grid, kProbeThreads, 0, s>>>(out, iters, 1.0f);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e == cudaSuccess && ms > 0.0f) {
    // two FMAs per packed instruction, two flops per FMA
    const double flops = (double)grid * kProbeThreads * iters * kProbeChains * 4.0;
    *tflops = flops / (ms * 1e-3) / 1e12;
  }
  if (out) cudaFree(out);
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (s) cudaStreamDestroy(s);
  return e;
}

}  // namespace cdvs
