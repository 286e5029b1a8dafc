// scfv.cu -- SCFV aggregation of an image's local descriptors into the
// global descriptor (Sec. III-D, Eq. 6-8; computed in the matrix-friendly
// form of Sec. IV-C, Eq. 9-14):
//
//   y_t        = P (x_t - m)                                   PCA 128 -> 32
//   gamma_t(i) = softmax_i( log w_i - 1/2 sum_k (y_tk - mu_ik)^2 / v_ik
//                           - 1/2 sum_k log(2 pi v_ik) )               Eq. 6, 9
//   g_mu(i)    = 1/(K sqrt(w_i))   sum_t gamma_t(i) (y_t - mu_i) / s_i  Eq. 7, 12
//   g_sigma(i) = 1/(K sqrt(2 w_i)) sum_t gamma_t(i) ((y_t - mu_i)^2/v_i - 1)   Eq. 13, 14
//   delta(i)   = population std of the 32 entries of g_mu(i)            Eq. 8
//
// then the components ranked by delta (descending, ties to the lower index)
// and the sign bits of g_mu for the first n_select of them.  Every sum runs
// in FP32 in a fixed order: the posterior is a softmax over 512 components of
// distances of ~32 terms, too sensitive for TF32 or BF16 operands, and the
// whole aggregation is ~30 MFLOP per image, so the FP32 pipes suffice.
#include <algorithm>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kComp = kScfvComp, kDim = kScfvDim, kIn = 128;

// K_a: y = P (x - m), one warp per record, lane j = output dimension j.
__global__ void __launch_bounds__(256) scfv_pca_kernel(const float* desc, int n_rec, const float* model,
                                                       float* Y) {
  __shared__ float pt[kIn * kDim];  // P transposed: [k][j]
  __shared__ float mean[kIn];
  for (int i = threadIdx.x; i < kIn * kDim; i += blockDim.x) pt[i] = model[kScfvOffPcaT + i];
  for (int i = threadIdx.x; i < kIn; i += blockDim.x) mean[i] = model[kScfvOffMean + i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rec; r += warps) {
    const float4 x4 = reinterpret_cast<const float4*>(desc + (size_t)r * kIn)[lane];
    const float x[4] = {x4.x - mean[4 * lane], x4.y - mean[4 * lane + 1], x4.z - mean[4 * lane + 2],
                        x4.w - mean[4 * lane + 3]};
    float acc = 0.0f;
    for (int q = 0; q < 32; ++q)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fmaf(__shfl_sync(0xffffffffu, x[c], q), pt[(4 * q + c) * kDim + lane], acc);
    Y[(size_t)r * kDim + lane] = acc;
  }
}

// K_b: posteriors of 32 records at a time; thread i = component i.
constexpr int kPostRec = 32;
__global__ void __launch_bounds__(kComp, 1) scfv_post_kernel(const float* Y, int n_rec, const float* model,
                                                             float* Q) {
  __shared__ __align__(16) float ys[kPostRec][kDim];
  __shared__ float red[kComp / 32][kPostRec];
  __shared__ float tot[kPostRec];
  const int i = threadIdx.x, lane = i & 31, warp = i >> 5;
  float mu[kDim], isd[kDim];
#pragma unroll
  for (int k = 0; k < kDim; ++k) {
    mu[k] = model[kScfvOffMu + i * kDim + k];
    isd[k] = model[kScfvOffIsd + i * kDim + k];
  }
  const float lw = model[kScfvOffLw + i];
  for (int r0 = blockIdx.x * kPostRec; r0 < n_rec; r0 += gridDim.x * kPostRec) {
    __syncthreads();
    for (int e = i; e < kPostRec * kDim; e += kComp) {
      const int r = e / kDim;
      ys[r][e - r * kDim] = r0 + r < n_rec ? Y[(size_t)(r0 + r) * kDim + e - r * kDim] : 0.0f;
    }
    __syncthreads();
    float l[kPostRec];
#pragma unroll
    for (int r = 0; r < kPostRec; ++r) {
      float d2 = 0.0f;
#pragma unroll
      for (int k = 0; k < kDim; k += 4) {
        const float4 y = *reinterpret_cast<const float4*>(&ys[r][k]);
        const float d0 = (y.x - mu[k]) * isd[k], d1 = (y.y - mu[k + 1]) * isd[k + 1];
        const float d2_ = (y.z - mu[k + 2]) * isd[k + 2], d3 = (y.w - mu[k + 3]) * isd[k + 3];
        d2 = fmaf(d0, d0, d2);
        d2 = fmaf(d1, d1, d2);
        d2 = fmaf(d2_, d2_, d2);
        d2 = fmaf(d3, d3, d2);
      }
      l[r] = fmaf(-0.5f, d2, lw);
    }
    // per record: max over the 512 components, then the sum of exponentials
#pragma unroll
    for (int r = 0; r < kPostRec; ++r) {
      float v = l[r];
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) red[warp][r] = v;
    }
    __syncthreads();
    if (i < kPostRec) {
      float v = red[0][i];
      for (int w = 1; w < kComp / 32; ++w) v = fmaxf(v, red[w][i]);
      tot[i] = v;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPostRec; ++r) {
      l[r] = expf(l[r] - tot[r]);
      float v = l[r];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][r] = v;
    }
    __syncthreads();
    if (i < kPostRec) {
      float v = 0.0f;
      for (int w = 0; w < kComp / 32; ++w) v += red[w][i];
      tot[i] = 1.0f / v;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPostRec; ++r)
      if (r0 + r < n_rec) Q[(size_t)(r0 + r) * kComp + i] = l[r] * tot[r];
  }
}

// K_c: Fisher gradients.  CTA = 32 components of one image; thread = one
// component and two dimensions.  Chunks of kGradRec records' posteriors (of
// those components) and projections are staged in shared memory with
// coalesced loads; every thread then sums its terms in record order.
constexpr int kGradComp = 32, kGradRec = 64, kGradThreads = 512;
__global__ void __launch_bounds__(kGradThreads) scfv_grad_kernel(const float* Y, const float* Q,
                                                                 const int* rec_off, const float* model,
                                                                 float* g_mu, float* g_sig) {
  __shared__ float qs[kGradRec][kGradComp];
  __shared__ float2 ys[kGradRec][kDim / 2];
  const int b = blockIdx.y, i0 = blockIdx.x * kGradComp;
  const int il = threadIdx.x >> 4, kp = threadIdx.x & 15;  // component i0 + il, dimensions 2 kp, 2 kp + 1
  const int i = i0 + il;
  const float2 mu = make_float2(model[kScfvOffMu + i * kDim + 2 * kp], model[kScfvOffMu + i * kDim + 2 * kp + 1]);
  const float2 isd = make_float2(model[kScfvOffIsd + i * kDim + 2 * kp], model[kScfvOffIsd + i * kDim + 2 * kp + 1]);
  const int t0 = rec_off[b], t1 = rec_off[b + 1];
  float a1x = 0.0f, a1y = 0.0f, a2x = 0.0f, a2y = 0.0f;
  for (int c0 = t0; c0 < t1; c0 += kGradRec) {
    const int nr = min(kGradRec, t1 - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < kGradRec * kGradComp; e += kGradThreads) {
      const int r = e / kGradComp, c = e - r * kGradComp;
      qs[r][c] = r < nr ? Q[(size_t)(c0 + r) * kComp + i0 + c] : 0.0f;
    }
    for (int e = threadIdx.x; e < kGradRec * (kDim / 2); e += kGradThreads) {
      const int r = e / (kDim / 2), c = e - r * (kDim / 2);
      ys[r][c] = r < nr ? reinterpret_cast<const float2*>(Y + (size_t)(c0 + r) * kDim)[c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      const float g = qs[r][il];
      const float2 y = ys[r][kp];
      const float dx = (y.x - mu.x) * isd.x, dy = (y.y - mu.y) * isd.y;
      a1x = fmaf(g, dx, a1x);
      a1y = fmaf(g, dy, a1y);
      a2x = fmaf(g, fmaf(dx, dx, -1.0f), a2x);
      a2y = fmaf(g, fmaf(dy, dy, -1.0f), a2y);
    }
  }
  const int K = t1 - t0;
  const float inv = K > 0 ? 1.0f / (float)K : 0.0f;
  const float nm = inv * model[kScfvOffNmu + i], ns = inv * model[kScfvOffNsig + i];
  const size_t o = ((size_t)b * kComp + i) * kDim + 2 * kp;
  reinterpret_cast<float2*>(g_mu + o)[0] = make_float2(a1x * nm, a1y * nm);
  reinterpret_cast<float2*>(g_sig + o)[0] = make_float2(a2x * ns, a2y * ns);
}

// K_d: delta, ranks and sign bits; one CTA per image, thread i = component i.
__global__ void __launch_bounds__(kComp) scfv_rank_kernel(const float* g_mu, int n_select, float* delta,
                                                          int* order, uint32_t* bits) {
  __shared__ float dl[kComp];
  const int b = blockIdx.x, i = threadIdx.x;
  const float4* g4 = reinterpret_cast<const float4*>(g_mu + ((size_t)b * kComp + i) * kDim);
  float v[kDim];
#pragma unroll
  for (int q = 0; q < kDim / 4; ++q) {
    const float4 x = g4[q];
    v[4 * q] = x.x;
    v[4 * q + 1] = x.y;
    v[4 * q + 2] = x.z;
    v[4 * q + 3] = x.w;
  }
  float mean = 0.0f;
#pragma unroll
  for (int k = 0; k < kDim; ++k) mean += v[k];
  mean *= 1.0f / kDim;
  float var = 0.0f;
#pragma unroll
  for (int k = 0; k < kDim; ++k) var = fmaf(v[k] - mean, v[k] - mean, var);
  const float d = sqrtf(var * (1.0f / kDim));
  dl[i] = d;
  __syncthreads();
  int rank = 0;
  for (int j = 0; j < kComp; ++j) rank += dl[j] > d || (dl[j] == d && j < i);
  delta[(size_t)b * kComp + i] = d;
  order[(size_t)b * kComp + rank] = i;
  if (rank < n_select) {
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < kDim; ++k) w |= (v[k] > 0.0f ? 1u : 0u) << k;
    bits[(size_t)b * n_select + rank] = w;
  }
}

}  // namespace

cudaError_t launch_scfv(const float* desc, int n_rec, const int* rec_off, int n_images, const float* model,
                        int n_select, float* Y, float* Q, float* g_mu, float* g_sig, float* delta, int* order,
                        uint32_t* bits, int n_sms, cudaStream_t s) {
  if (n_images <= 0) return cudaSuccess;
  if (n_rec > 0) {
    scfv_pca_kernel<<<std::max(1, std::min((n_rec + 7) / 8, n_sms * 8)), 256, 0, s>>>(desc, n_rec, model, Y);
    scfv_post_kernel<<<std::max(1, std::min((n_rec + kPostRec - 1) / kPostRec, n_sms)), kComp, 0, s>>>(Y, n_rec,
                                                                                                   model, Q);
  }
  scfv_grad_kernel<<<dim3(kComp / kGradComp, n_images), kGradThreads, 0, s>>>(Y, Q, rec_off, model, g_mu, g_sig);
  scfv_rank_kernel<<<n_images, kComp, 0, s>>>(g_mu, n_select, delta, order, bits);
  return cudaGetLastError();
}

}  // namespace cdvs
