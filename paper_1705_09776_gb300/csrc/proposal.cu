// proposal.cu -- the learned block proposal: a small CNN that gives one logit
// per 16x16 block of an 8-bit image, trained on blocks that hold interest
// points of the plain detector (ALP, Sec. IV-A), so that detection can skip
// blocks where none is likely.
//
//   x  = (u8 - 128) / 64
//   A1 = relu(conv3x3(x,  W1, stride 2) + b1)      16 ch, BF16
//   A2 = relu(conv3x3(A1, W2, stride 2) + b2)      16 ch, BF16
//   A3 = relu(conv3x3(A2, W3, stride 1) + b3)      16 ch, FP32
//   z  = Wh . mean_4x4(A3) + bh                    one logit per 16x16 block
//
// (padding 1 everywhere; weights used in BF16, biases and every accumulation
// in FP32).  Two implementations of the forward pass:
//  * training kernels, one per layer, on the FP32 pipes with the BF16
//    roundings applied where the network stores BF16 (bf16 = 0 turns them
//    off for gradient checks), followed by the backward kernels, the BCE
//    loss and Adam; every reduction runs in a fixed order, so a training
//    step is deterministic;
//  * the fused inference kernel: one CTA per 8x4 blocks keeps the input,
//    A1 and A2 of its region in shared memory; conv2 and conv3 are 9
//    contractions (one per tap) of K = 16 input channels on the tensor cores
//    (mma.sync m16n8k16 BF16 -> FP32), and each conv3 row tile of 16
//    positions is exactly one 4x4 pooling cell, so the pooling is a warp
//    reduction.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kC = 16;
constexpr int kOffW1 = 0, kOffB1 = 144, kOffW2 = 160, kOffB2 = 2464, kOffW3 = 2480, kOffB3 = 4784,
              kOffWh = 4800, kOffBh = 4816;
static_assert(kOffBh + 1 == kPropParams, "parameter layout");

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float wq(const float* theta, int i, int bf16) { return bf16 ? bf16r(theta[i]) : theta[i]; }

// ------------------------------------------------------------------ training
// Activations are planar FP32 tensors [B][16][H][W] (A1, A2 hold BF16 values
// in bf16 mode).  A > 0 exactly where the pre-activation was > 0, so the
// ReLU masks of the backward pass come from the stored activations.

struct U8Input {  // the network input x = (u8 - 128) / 64, zero outside
  const uint8_t* img;
  int pitch;
  size_t stride;  // bytes between images
  int H, W;
  __device__ __forceinline__ float operator()(int b, int ci, int y, int x) const {
    (void)ci;
    if (y < 0 || y >= H || x < 0 || x >= W) return 0.0f;
    return ((float)img[(size_t)b * stride + (size_t)y * pitch + x] - 128.0f) * (1.0f / 64.0f);
  }
};

struct F32Input {  // planar [B][C][H][W], zero outside
  const float* a;
  int C, H, W;
  __device__ __forceinline__ float operator()(int b, int ci, int y, int x) const {
    if (y < 0 || y >= H || x < 0 || x >= W) return 0.0f;
    return a[(((size_t)b * C + ci) * H + y) * W + x];
  }
};

// Forward of one 3x3 layer with CIN inputs and 16 outputs, stride S: one
// thread per output pixel, all 16 channels.  round_out: BF16 activations.
template <int CIN, int S, typename In>
__global__ void __launch_bounds__(256) conv_fwd_kernel(In in, const float* theta, int w_off, int b_off, int bf16,
                                                       int round_out, float* out, int B, int Ho, int Wo) {
  __shared__ float w[kC * CIN * 9];
  __shared__ float bias[kC];
  for (int i = threadIdx.x; i < kC * CIN * 9; i += blockDim.x) w[i] = wq(theta, w_off + i, bf16);
  if (threadIdx.x < kC) bias[threadIdx.x] = theta[b_off + threadIdx.x];
  __syncthreads();
  const long long n = (long long)B * Ho * Wo;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / ((long long)Ho * Wo));
    const int r = (int)(idx - (long long)b * Ho * Wo);
    const int y = r / Wo, x = r - (r / Wo) * Wo;
    float acc[kC];
#pragma unroll
    for (int co = 0; co < kC; ++co) acc[co] = bias[co];
    for (int ci = 0; ci < CIN; ++ci)
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float v = in(b, ci, S * y + k / 3 - 1, S * x + k % 3 - 1);
#pragma unroll
        for (int co = 0; co < kC; ++co) acc[co] = fmaf(w[(co * CIN + ci) * 9 + k], v, acc[co]);
      }
#pragma unroll
    for (int co = 0; co < kC; ++co) {
      float a = fmaxf(acc[co], 0.0f);
      if (round_out) a = bf16r(a);
      out[(((size_t)b * kC + co) * Ho + y) * Wo + x] = a;
    }
  }
}

// Pooling, head and loss, one thread per block: P (kept for the head
// gradient), the logit z, dL/dz = (sigmoid(z) - y) / n_blocks and the
// block's loss softplus(z) - y z; per-CTA loss sums in a fixed tree order.
__global__ void __launch_bounds__(256) pool_head_kernel(const float* a3, int B, int H2, int W2, int Th, int Tw,
                                                        const float* theta, int bf16, const float* labels,
                                                        float* P, float* z_out, float* dz, float* loss_part) {
  __shared__ float red[256];
  const int n = B * Th * Tw;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (i < n) {
    const int b = i / (Th * Tw), t = i - b * Th * Tw, ty = t / Tw, tx = t - (t / Tw) * Tw;
    const int y0 = 4 * ty, x0 = 4 * tx, y1 = min(y0 + 4, H2), x1 = min(x0 + 4, W2);
    const int cnt = max(y1 - y0, 0) * max(x1 - x0, 0);
    float z = theta[kOffBh];
    for (int c = 0; c < kC; ++c) {
      float s = 0.0f;
      for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) s += a3[(((size_t)b * kC + c) * H2 + y) * W2 + x];
      const float p = cnt > 0 ? s / (float)cnt : 0.0f;
      P[(size_t)i * kC + c] = p;
      z = fmaf(wq(theta, kOffWh + c, bf16), p, z);
    }
    z_out[i] = z;
    if (labels) {
      const float y = labels[i];
      dz[i] = (1.0f / (1.0f + expf(-z)) - y) / (float)n;
      l = fmaxf(z, 0.0f) - y * z + log1pf(expf(-fabsf(z)));
    }
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// dL/dZ3 = [A3 > 0] Wh[c] dz(block) / count(block)
__global__ void __launch_bounds__(256) dz3_kernel(const float* a3, const float* dz, const float* theta, int bf16,
                                                  int B, int H2, int W2, int Th, int Tw, float* dz3) {
  const long long n = (long long)B * kC * H2 * W2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(idx % W2);
    const int y = (int)((idx / W2) % H2);
    const int c = (int)((idx / ((long long)W2 * H2)) % kC);
    const int b = (int)(idx / ((long long)W2 * H2 * kC));
    const int ty = y / 4, tx = x / 4;
    const int cnt = (min(4 * ty + 4, H2) - 4 * ty) * (min(4 * tx + 4, W2) - 4 * tx);
    const float g = wq(theta, kOffWh + c, bf16) * dz[((size_t)b * Th + ty) * Tw + tx] / (float)cnt;
    dz3[idx] = a3[idx] > 0.0f ? g : 0.0f;
  }
}

// Input gradient of a 16 -> 16 layer of stride S, times the ReLU mask of its
// input: dZin[ci](y, x) = [Ain > 0] sum over co, taps with S yo + ky - 1 = y
// (and the same in x) of dZ[co](yo, xo) W[co][ci][ky][kx].
template <int S>
__global__ void __launch_bounds__(256) conv_dgrad_kernel(const float* dz, int Ho, int Wo, const float* ain, int Hi,
                                                         int Wi, const float* theta, int w_off, int bf16, int B,
                                                         float* dzin) {
  __shared__ float w[kC * kC * 9];
  for (int i = threadIdx.x; i < kC * kC * 9; i += blockDim.x) w[i] = wq(theta, w_off + i, bf16);
  __syncthreads();
  const long long n = (long long)B * Hi * Wi;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / ((long long)Hi * Wi));
    const int r = (int)(idx - (long long)b * Hi * Wi);
    const int y = r / Wi, x = r - (r / Wi) * Wi;
    float acc[kC];
#pragma unroll
    for (int ci = 0; ci < kC; ++ci) acc[ci] = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ty = y + 1 - k / 3, tx = x + 1 - k % 3;
      if (ty < 0 || tx < 0 || ty % S || tx % S) continue;
      const int yo = ty / S, xo = tx / S;
      if (yo >= Ho || xo >= Wo) continue;
      for (int co = 0; co < kC; ++co) {
        const float g = dz[(((size_t)b * kC + co) * Ho + yo) * Wo + xo];
#pragma unroll
        for (int ci = 0; ci < kC; ++ci) acc[ci] = fmaf(w[(co * kC + ci) * 9 + k], g, acc[ci]);
      }
    }
#pragma unroll
    for (int ci = 0; ci < kC; ++ci) {
      const size_t o = (((size_t)b * kC + ci) * Hi + y) * Wi + x;
      dzin[o] = ain[o] > 0.0f ? acc[ci] : 0.0f;
    }
  }
}

// Weight and bias gradients of a CIN -> 16 layer of stride S.  Each CTA takes
// chunks of 64 output pixels (grid-stride, so the assignment is fixed), stages
// their dZ and input patches, and thread j accumulates the weights j,
// j + 256, ...; per-CTA partial sums go to part[blockIdx.x][16 * CIN * 9 + 16].
constexpr int kWgChunk = 64;
template <int CIN, int S, typename In>
__global__ void __launch_bounds__(256) conv_wgrad_kernel(In in, const float* dz, int B, int Ho, int Wo,
                                                         float* part) {
  constexpr int NW = kC * CIN * 9, PL = CIN * 9;
  __shared__ float sdz[kC][kWgChunk];
  __shared__ float patch[kWgChunk][PL + 1];
  float acc[(NW + 255) / 256];
  float bacc = 0.0f;
#pragma unroll
  for (int m = 0; m < (NW + 255) / 256; ++m) acc[m] = 0.0f;
  const long long n = (long long)B * Ho * Wo;
  for (long long c0 = (long long)blockIdx.x * kWgChunk; c0 < n; c0 += (long long)gridDim.x * kWgChunk) {
    __syncthreads();
    for (int i = threadIdx.x; i < kWgChunk * (kC + PL); i += blockDim.x) {
      const int p = i % kWgChunk, f = i / kWgChunk;
      const long long idx = c0 + p;
      float v = 0.0f;
      if (idx < n) {
        const int b = (int)(idx / ((long long)Ho * Wo));
        const int r = (int)(idx - (long long)b * Ho * Wo);
        const int y = r / Wo, x = r - (r / Wo) * Wo;
        if (f < kC) {
          v = dz[(((size_t)b * kC + f) * Ho + y) * Wo + x];
        } else {
          const int ci = (f - kC) / 9, k = (f - kC) % 9;
          v = in(b, ci, S * y + k / 3 - 1, S * x + k % 3 - 1);
        }
      }
      if (f < kC) sdz[f][p] = v;
      else patch[p][f - kC] = v;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < (NW + 255) / 256; ++m) {
      const int j = threadIdx.x + 256 * m;
      if (j < NW) {
        const int co = j / PL, q = j - co * PL;
        float s = acc[m];
        for (int p = 0; p < kWgChunk; ++p) s = fmaf(sdz[co][p], patch[p][q], s);
        acc[m] = s;
      }
    }
    if (threadIdx.x < kC)
      for (int p = 0; p < kWgChunk; ++p) bacc += sdz[threadIdx.x][p];
  }
  float* out = part + (size_t)blockIdx.x * (NW + kC);
#pragma unroll
  for (int m = 0; m < (NW + 255) / 256; ++m) {
    const int j = threadIdx.x + 256 * m;
    if (j < NW) out[j] = acc[m];
  }
  if (threadIdx.x < kC) out[NW + threadIdx.x] = bacc;
}

// grad[w_off + j] = sum over g of part[g][j] (j < nw), grad[b_off + c] from
// the bias columns; g in increasing order.
__global__ void reduce_parts_kernel(const float* part, int n_parts, int nw, float* grad, int w_off, int b_off) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nw + kC) return;
  float s = 0.0f;
  for (int g = 0; g < n_parts; ++g) s += part[(size_t)g * (nw + kC) + j];
  grad[j < nw ? w_off + j : b_off + (j - nw)] = s;
}

// Head gradients (one CTA per output: dWh[c] = sum dz P[c], dbh = sum dz) and,
// in the CTA of bh, the mean loss from the pool kernel's CTA sums.
__global__ void __launch_bounds__(256) head_grad_kernel(const float* P, const float* dz, int n, float* grad,
                                                        const float* loss_part, int n_loss, float* loss) {
  __shared__ float red[256];
  const int c = blockIdx.x;  // 0..15 weights, 16 bias
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += dz[i] * (c < kC ? P[(size_t)i * kC + c] : 1.0f);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad[c < kC ? kOffWh + c : kOffBh] = red[0];
  if (c == kC && threadIdx.x == 0 && loss) {
    float l = 0.0f;
    for (int g = 0; g < n_loss; ++g) l += loss_part[g];
    *loss = l / (float)n;
  }
}

// Adam with bias correction: bc1 = 1 - beta1^t, bc2 = 1 - beta2^t.
__global__ void adam_kernel(float* theta, float* m, float* v, const float* g, int n, float lr, float b1, float b2,
                            float bc1, float bc2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ------------------------------------------------------------------ inference
constexpr int kRBX = 8, kRBY = 4;                          // blocks per CTA
constexpr int kA3X = 4 * kRBX, kA3Y = 4 * kRBY;            // 32 x 16 A3 positions
constexpr int kA2X = kA3X + 2, kA2Y = kA3Y + 2;            // 34 x 18 (conv3 halo)
constexpr int kA1X = 2 * kA2X + 1, kA1Y = 2 * kA2Y + 1;    // 69 x 37
constexpr int kInX = 2 * kA1X + 1, kInY = 2 * kA1Y + 1;    // 139 x 75
constexpr int kInP = 160;                                  // input row pitch (bytes): 139 + 15 alignment slack
constexpr int kInfThreads = 256;
static_assert(kInX + 15 <= kInP, "input rows hold the region after 16-byte alignment");
constexpr int kA2Tiles = (kA2X * kA2Y + 15) / 16;          // 39 row tiles of conv2
// Shared-memory layout of the activations: one position holds 16 BF16
// channels in two 16-byte chunks (channels 0-7, 8-15), chunk index 2 p + half.
// Both buffers permute chunks within each 128-byte line (8 chunks) by an XOR
// swizzle so that the 8 rows of every ldmatrix matrix fall in 8 different
// bank groups:
//  * A1 (row pitch 69 positions): conv2 reads positions two apart, so chunk
//    bits 0-1 are XORed with bits 3-4;
//  * A2 (row pitch 36 positions, 34 used): conv3 reads two runs of 4
//    positions one row apart, so chunk bit 0 is XORed with bit 3.
// Each buffer is a whole number of lines, so a swizzled chunk stays inside it.
constexpr int kA2P = 36;                                   // A2 row pitch in shared memory (positions)
constexpr size_t kLine = 128;
constexpr size_t kInBytes = ((size_t)kInY * kInP + kLine - 1) / kLine * kLine;
constexpr size_t kA1Bytes = ((size_t)kA1X * kA1Y * kC * 2 + kLine - 1) / kLine * kLine;
constexpr size_t kA2Bytes = ((size_t)kA2P * kA2Y * kC * 2 + kLine - 1) / kLine * kLine;
constexpr size_t kInfSmem = kInBytes + kA1Bytes + kA2Bytes;
// two CTAs per SM: 228 KB per SM, each CTA also holds under 1 KB of static
// arrays and the 1 KB the hardware reserves
static_assert(2 * (kInfSmem + 1024 + 1024) <= 228 * 1024, "two CTAs per SM");
__device__ __forceinline__ int a1_chunk(int c) { return c ^ ((c >> 3) & 3); }
__device__ __forceinline__ int a2_chunk(int c) { return c ^ ((c >> 3) & 1); }

__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half)
  return *reinterpret_cast<const unsigned*>(&v);
}
// relu, round to BF16 and pack in one instruction (the first source goes to
// the upper half)
__device__ __forceinline__ unsigned pack_relu_bf16(float lo, float hi) {
  unsigned r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// B fragments of one 16 -> 16 layer for this lane, prepacked by the host
// (pack_proposal_fragments): one coalesced 8-byte load per tap and half.
__device__ __forceinline__ void load_bfrag(const uint2* frag, int layer, int lane, unsigned (&bw)[9][2][2]) {
#pragma unroll
  for (int t = 0; t < 9; ++t)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint2 v = frag[((layer * 9 + t) * 2 + h) * 32 + lane];
      bw[t][h][0] = v.x;
      bw[t][h][1] = v.y;
    }
}

__global__ void __launch_bounds__(kInfThreads, 2) proposal_infer_kernel(const PropImage* imgs, const float* theta,
                                                                        const uint2* frag, float* logits) {
  extern __shared__ float4 smem4[];
  uint8_t* in_s = reinterpret_cast<uint8_t*>(smem4);
  __nv_bfloat16* a1_s = reinterpret_cast<__nv_bfloat16*>(in_s + kInBytes);
  __nv_bfloat16* a2_s = reinterpret_cast<__nv_bfloat16*>(in_s + kInBytes + kA1Bytes);
  __shared__ float w1[kC * 9], b1[kC], b2[kC], b3[kC], wh[kC];
  const PropImage im = imgs[blockIdx.z];
  const int bx0 = blockIdx.x * kRBX, by0 = blockIdx.y * kRBY;  // first block of the CTA
  if (bx0 >= im.Tw || by0 >= im.Th) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // global origins of the regions (A3, A2, A1, input)
  const int ya3 = 4 * by0, xa3 = 4 * bx0;
  const int ya2 = ya3 - 1, xa2 = xa3 - 1;
  const int ya1 = 2 * ya2 - 1, xa1 = 2 * xa2 - 1;
  const int yin = 2 * ya1 - 1, xin = 2 * xa1 - 1;
  for (int i = threadIdx.x; i < kC * 9; i += kInfThreads) w1[i] = bf16r(theta[kOffW1 + i]);
  if (threadIdx.x < kC) {
    b1[threadIdx.x] = theta[kOffB1 + threadIdx.x];
    b2[threadIdx.x] = theta[kOffB2 + threadIdx.x];
    b3[threadIdx.x] = theta[kOffB3 + threadIdx.x];
    wh[threadIdx.x] = bf16r(theta[kOffWh + threadIdx.x]);
  }
  // input region, from image column xal = xin rounded down to 16 bytes (so
  // in_s column c + sh is image x = xin + c): 16-byte asynchronous copies of
  // the aligned pieces inside the image, bytes elsewhere (128 = x of 0
  // outside the image: the zero padding of x)
  const int xal = xin & ~15, sh = xin - xal;
  const bool vec = ((reinterpret_cast<uintptr_t>(im.src) | (uintptr_t)im.pitch) & 15) == 0;
  for (int i = threadIdx.x; i < kInY * (kInP / 16); i += kInfThreads) {
    const int r = i / (kInP / 16), c16 = i - r * (kInP / 16);
    const int gy = yin + r, gx = xal + 16 * c16;
    uint8_t* dst = in_s + r * kInP + 16 * c16;
    if (vec && gy >= 0 && gy < im.H && gx >= 0 && gx + 16 <= im.W) {
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                       static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                   "l"(im.src + (size_t)gy * im.pitch + gx)
                   : "memory");
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int x = gx + j;
        dst[j] = (gy >= 0 && gy < im.H && x >= 0 && x < im.W) ? im.src[(size_t)gy * im.pitch + x] : 128;
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // conv1 on the tensor cores: row tiles of 16 A1 positions (row-major over
  // the 69 x 37 region) times the 9 taps (K padded to 16 with zeros) -> 16
  // channels, mma.sync m16n8k16 BF16 -> FP32.  The inputs (u8 - 128) / 64
  // are exact in BF16 and the weights are BF16-rounded, so every product is
  // exact; A1 is zero outside the layer.  Fragments (lane = 4 g + t): A
  // register q holds position g + 8 (q & 1), taps 2t + 8 (q >> 1) + {0, 1};
  // B register q holds taps 2t + 8q + {0, 1}, channel 8h + g; C holds
  // positions g, g + 8 and channels 8h + 2t + {0, 1}.
  {
    const int g = lane >> 2, t = lane & 3;
    unsigned bw1[2][2];  // [n-tile h][register q]
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k0 = 2 * t + 8 * q, co = 8 * h + g;
        const float w0 = k0 < 9 ? w1[co * 9 + k0] : 0.0f, wv = k0 + 1 < 9 ? w1[co * 9 + k0 + 1] : 0.0f;
        bw1[h][q] = pack_bf16(w0, wv);
      }
    float bias[2][2];  // this lane's output channels 8 h + 2 t + {0, 1}
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      bias[h][0] = b1[8 * h + 2 * t];
      bias[h][1] = b1[8 * h + 2 * t + 1];
    }
    constexpr int kA1N = kA1X * kA1Y, kA1Tiles = (kA1N + 15) / 16;
    for (int tile = warp; tile < kA1Tiles; tile += kInfThreads / 32) {
      int pr[2], rr1[2], cc1[2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        pr[hh] = 16 * tile + g + 8 * hh;
        const int pc = min(pr[hh], kA1N - 1);  // past the region: a valid position, not stored
        rr1[hh] = pc / kA1X;
        cc1[hh] = pc - rr1[hh] * kA1X;
      }
      auto x = [&](int hh, int k) {  // input of tap k for position hh (k < 9)
        return ((float)in_s[(2 * rr1[hh] + k / 3) * kInP + sh + 2 * cc1[hh] + k % 3] - 128.0f) * (1.0f / 64.0f);
      };
      unsigned a[4];
      a[0] = pack_bf16(x(0, 2 * t), x(0, 2 * t + 1));
      a[1] = pack_bf16(x(1, 2 * t), x(1, 2 * t + 1));
      a[2] = t == 0 ? pack_bf16(x(0, 8), 0.0f) : 0u;
      a[3] = t == 0 ? pack_bf16(x(1, 8), 0.0f) : 0u;
      // accumulators start at the bias
      float acc[2][4] = {{bias[0][0], bias[0][1], bias[0][0], bias[0][1]},
                         {bias[1][0], bias[1][1], bias[1][0], bias[1][1]}};
      mma_bf16(acc[0], a, bw1[0][0], bw1[0][1]);
      mma_bf16(acc[1], a, bw1[1][0], bw1[1][1]);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int p = pr[hh];
        if (p >= kA1N) continue;
        const int gy = ya1 + rr1[hh], gx = xa1 + cc1[hh];
        const bool ok = gy >= 0 && gy < im.H1 && gx >= 0 && gx < im.W1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned v = pack_relu_bf16(acc[h][2 * hh], acc[h][2 * hh + 1]);
          reinterpret_cast<unsigned*>(a1_s)[4 * a1_chunk(2 * p + h) + t] = ok ? v : 0u;
        }
      }
    }
  }
  __syncthreads();
  const int q = lane & 3, rr = lane >> 2;
  // conv2 on the tensor cores: row tiles of 16 A2 positions (row-major over
  // the 34 x 18 region), one K = 16 contraction per tap
  {
    unsigned bw[9][2][2];
    load_bfrag(frag, 0, lane, bw);
    float bias[2][2];  // this lane's output channels 8 h + 2 q + {0, 1}
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      bias[h][0] = b2[8 * h + 2 * q];
      bias[h][1] = b2[8 * h + 2 * q + 1];
    }
    for (int t = warp; t < kA2Tiles; t += kInfThreads / 32) {
      // this lane's ldmatrix row: position 16 t + lane % 16 (clamped), k half lane / 16
      const int pr = min(16 * t + (lane & 15), kA2X * kA2Y - 1);
      const int r2 = pr / kA2X, c2 = pr - (pr / kA2X) * kA2X;
      const int c0 = 2 * ((2 * r2) * kA1X + 2 * c2) + (lane >> 4);  // chunk of tap 0
      // accumulators start at the bias
      float acc[2][4] = {{bias[0][0], bias[0][1], bias[0][0], bias[0][1]},
                         {bias[1][0], bias[1][1], bias[1][0], bias[1][1]}};
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        unsigned a[4];
        ldmatrix_x4(a, a1_s + 8 * a1_chunk(c0 + 2 * ((k / 3) * kA1X + k % 3)));
        mma_bf16(acc[0], a, bw[k][0][0], bw[k][0][1]);
        mma_bf16(acc[1], a, bw[k][1][0], bw[k][1][1]);
      }
#pragma unroll
      for (int half = 0; half < 2; ++half) {  // rows rr and rr + 8
        const int p = 16 * t + rr + 8 * half;
        if (p >= kA2X * kA2Y) continue;
        const int r2o = p / kA2X, c2o = p - (p / kA2X) * kA2X;
        const int gy = ya2 + r2o, gx = xa2 + c2o;
        const bool ok = gy >= 0 && gy < im.H2 && gx >= 0 && gx < im.W2;
        const int ps = r2o * kA2P + c2o;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned v = pack_relu_bf16(acc[h][2 * half], acc[h][2 * half + 1]);
          reinterpret_cast<unsigned*>(a2_s)[4 * a2_chunk(2 * ps + h) + q] = ok ? v : 0u;
        }
      }
    }
  }
  __syncthreads();
  // conv3 + pooling + head: row tile t = pooling cell (t / 8, t % 8) of the
  // CTA, row i = position (4 (t / 8) + i / 4, 4 (t % 8) + i % 4)
  {
    unsigned bw[9][2][2];
    load_bfrag(frag, 1, lane, bw);
    for (int t = warp; t < kRBX * kRBY; t += kInfThreads / 32) {
      const int cy = t / kRBX, cx = t - (t / kRBX) * kRBX;
      const int ty = by0 + cy, tx = bx0 + cx;
      if (ty >= im.Th || tx >= im.Tw) continue;  // warp-uniform
      const int i = lane & 15;
      const int r3 = 4 * cy + i / 4, c3 = 4 * cx + i % 4;
      const int c0 = 2 * (r3 * kA2P + c3) + (lane >> 4);  // chunk of tap 0
      float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        unsigned a[4];
        ldmatrix_x4(a, a2_s + 8 * a2_chunk(c0 + 2 * ((k / 3) * kA2P + k % 3)));
        mma_bf16(acc[0], a, bw[k][0][0], bw[k][0][1]);
        mma_bf16(acc[1], a, bw[k][1][0], bw[k][1][1]);
      }
      // relu(z3 + b3) at the lane's two rows, zero for positions outside A3
      float s[2][2];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 2; ++j) s[h][j] = 0.0f;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int ii = rr + 8 * half;
        const int gy = ya3 + 4 * cy + ii / 4, gx = xa3 + 4 * cx + ii % 4;
        if (gy < im.H2 && gx < im.W2)
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 2; ++j) s[h][j] += fmaxf(acc[h][2 * half + j] + b3[8 * h + 2 * q + j], 0.0f);
      }
      // sum over the 8 row lanes (same q): lane bits 2..4
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int o = 4; o < 32; o <<= 1) s[h][j] += __shfl_xor_sync(0xffffffffu, s[h][j], o);
      const int gy0 = 4 * ty, gx0 = 4 * tx;
      const int cnt = (min(gy0 + 4, im.H2) - gy0) * (min(gx0 + 4, im.W2) - gx0);
      const float inv = 1.0f / (float)cnt;
      float zp = 0.0f;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 2; ++j) zp = fmaf(wh[8 * h + 2 * q + j], s[h][j] * inv, zp);
      zp += __shfl_xor_sync(0xffffffffu, zp, 1);
      zp += __shfl_xor_sync(0xffffffffu, zp, 2);
      if (lane == 0) logits[im.logit_off + (size_t)ty * im.Tw + tx] = zp + theta[kOffBh];
    }
  }
}

// Tile modes of the first octave, in three passes over the batch.
// near[block]: a block with logit > zt lies within `dil` blocks.
__global__ void near_kernel(const PropImage* imgs, int n_images, const float* logits, float zt, int dil,
                            uint8_t* near) {
  const int img = blockIdx.y;
  if (img >= n_images) return;
  const PropImage im = imgs[img];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < im.Th * im.Tw; i += gridDim.x * blockDim.x) {
    const int by = i / im.Tw, bx = i - (i / im.Tw) * im.Tw;
    bool hit = false;
    for (int yy = max(by - dil, 0); yy <= min(by + dil, im.Th - 1); ++yy)
      for (int xx = max(bx - dil, 0); xx <= min(bx + dil, im.Tw - 1); ++xx)
        hit |= logits[im.logit_off + (size_t)yy * im.Tw + xx] > zt;
    near[im.logit_off + i] = hit;
  }
}

// Per first-octave tile (128 x 32 px = 8 x 2 blocks): block_mask = its near
// blocks (bit 8 row + col), det = any of them.
__global__ void tile_det_kernel(const PropImage* imgs, const ImgPlan* plans, const int* tile_prefix, int n_images,
                                const uint8_t* near, uint16_t* block_mask, uint8_t* det) {
  const int img = blockIdx.y;
  if (img >= n_images) return;
  const PropImage im = imgs[img];
  const OctPlan& op = plans[img].oct[0];
  constexpr int bw = kTX / 16, bh = kTY / 16;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < op.tiles_x * op.tiles_y; t += gridDim.x * blockDim.x) {
    const int ty = t / op.tiles_x, tx = t - ty * op.tiles_x;
    unsigned bits = 0;
#pragma unroll
    for (int j = 0; j < bw * bh; ++j) {
      const int by = ty * bh + j / bw, bx = tx * bw + j % bw;
      if (by < im.Th && bx < im.Tw && near[im.logit_off + (size_t)by * im.Tw + bx]) bits |= 1u << j;
    }
    block_mask[tile_prefix[img] + t] = (uint16_t)bits;
    det[tile_prefix[img] + t] = bits != 0;
  }
}

// mode: kModeDetect for detecting tiles, kModeLevels when a detecting tile
// lies within (ny, nx) tiles (a descriptor disc of its points may read this
// tile's levels), else kModeLevel3.
__global__ void tile_mode_kernel(const ImgPlan* plans, const int* tile_prefix, int n_images, const uint8_t* det,
                                 int ny, int nx, uint8_t* mode) {
  const int img = blockIdx.y;
  if (img >= n_images) return;
  const OctPlan& op = plans[img].oct[0];
  const uint8_t* d = det + tile_prefix[img];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < op.tiles_x * op.tiles_y; t += gridDim.x * blockDim.x) {
    const int ty = t / op.tiles_x, tx = t - ty * op.tiles_x;
    uint8_t m = kModeLevel3;
    if (d[t]) {
      m = kModeDetect;
    } else {
      bool any = false;
      for (int uy = max(ty - ny, 0); uy <= min(ty + ny, op.tiles_y - 1); ++uy)
        for (int ux = max(tx - nx, 0); ux <= min(tx + nx, op.tiles_x - 1); ++ux) any |= d[uy * op.tiles_x + ux] != 0;
      if (any) m = kModeLevels;
    }
    mode[tile_prefix[img] + t] = m;
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers
size_t proposal_infer_smem() { return kInfSmem; }

// The B fragments of conv2 (layer 0) and conv3 (layer 1) for every lane:
// frag[((layer 9 + t) 2 + h) 32 + lane] = {W[co][2q, 2q + 1][t], W[co][2q + 8, 2q + 9][t]} in BF16 (round to
// nearest even, low half = lower ci), co = 8h + lane / 4, q = lane % 4: the register layout of the B operand of
// mma.m16n8k16 (.col).  n = kPropFragWords uint32 words.
void pack_proposal_fragments(const float* theta, uint32_t* frag) {
  auto bits = [](float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;  // BF16, round to nearest even
  };
  const int w_off[2] = {kOffW2, kOffW3};
  for (int layer = 0; layer < 2; ++layer)
    for (int t = 0; t < 9; ++t)
      for (int h = 0; h < 2; ++h)
        for (int lane = 0; lane < 32; ++lane) {
          const int q = lane & 3, co = 8 * h + (lane >> 2);
          const float* w = theta + w_off[layer] + co * kC * 9 + t;
          uint32_t* o = frag + 2 * (((layer * 9 + t) * 2 + h) * 32 + lane);
          o[0] = bits(w[(2 * q) * 9]) | (bits(w[(2 * q + 1) * 9]) << 16);
          o[1] = bits(w[(2 * q + 8) * 9]) | (bits(w[(2 * q + 9) * 9]) << 16);
        }
}

cudaError_t launch_proposal_infer(const PropImage* d_imgs, int n_images, int max_th, int max_tw, const float* theta,
                                  const uint32_t* frag, float* logits, cudaStream_t s) {
  if (n_images <= 0) return cudaSuccess;
  static LaunchCache cache;
  cudaError_t e = prepare_launch(proposal_infer_kernel, cache, (int)kInfSmem, kInfThreads, nullptr);
  if (e != cudaSuccess) return e;
  dim3 grid((max_tw + kRBX - 1) / kRBX, (max_th + kRBY - 1) / kRBY, n_images);
  proposal_infer_kernel<<<grid, kInfThreads, kInfSmem, s>>>(d_imgs, theta, reinterpret_cast<const uint2*>(frag),
                                                            logits);
  return cudaGetLastError();
}

// scratch: max(n_logits, 1) + n_tiles bytes
cudaError_t launch_tile_mode(const PropImage* d_imgs, const ImgPlan* plans, const int* tile_prefix, int n_images,
                             int max_blocks, int max_tiles, const float* logits, float zt, int dil, int ny, int nx,
                             uint8_t* mode, uint16_t* block_mask, uint8_t* near, uint8_t* det, cudaStream_t s) {
  if (n_images <= 0) return cudaSuccess;
  near_kernel<<<dim3((max_blocks + 255) / 256, n_images), 256, 0, s>>>(d_imgs, n_images, logits, zt, dil, near);
  tile_det_kernel<<<dim3((max_tiles + 127) / 128, n_images), 128, 0, s>>>(d_imgs, plans, tile_prefix, n_images, near,
                                                                        block_mask, det);
  tile_mode_kernel<<<dim3((max_tiles + 127) / 128, n_images), 128, 0, s>>>(plans, tile_prefix, n_images, det, ny, nx,
                                                                         mode);
  return cudaGetLastError();
}

// Workspace layout of a training step (floats): A1, A2, A3, dZ1, dZ2, dZ3,
// P, z, dz, loss parts, weight-gradient parts.
size_t proposal_train_floats(int B, int H, int W, int n_sms) {
  const size_t H1 = (H + 1) / 2, W1 = (W + 1) / 2, H2 = (H1 + 1) / 2, W2 = (W1 + 1) / 2;
  const size_t Th = (H + 15) / 16, Tw = (W + 15) / 16;
  const size_t a1 = (size_t)B * kC * H1 * W1, a2 = (size_t)B * kC * H2 * W2;
  const size_t nb = (size_t)B * Th * Tw;
  const size_t parts = (size_t)2 * n_sms * (kC * kC * 9 + kC);
  return 2 * a1 + 4 * a2 + nb * kC + 2 * nb + (nb + 255) / 256 + parts;
}

cudaError_t run_proposal_train(const PropTrainArgs& t, float* ws, int n_sms, cudaStream_t s) {
  const int B = t.B, H = t.H, W = t.W;
  const int H1 = (H + 1) / 2, W1 = (W + 1) / 2, H2 = (H1 + 1) / 2, W2 = (W1 + 1) / 2;
  const int Th = (H + 15) / 16, Tw = (W + 15) / 16;
  const size_t na1 = (size_t)B * kC * H1 * W1, na2 = (size_t)B * kC * H2 * W2;
  const int nb = B * Th * Tw;
  float* a1 = ws;
  float* dz1 = a1 + na1;
  float* a2 = dz1 + na1;
  float* dz2 = a2 + na2;
  float* a3 = dz2 + na2;
  float* dz3 = a3 + na2;
  float* P = dz3 + na2;
  float* z = P + (size_t)nb * kC;
  float* dz = z + nb;
  float* lpart = dz + nb;
  const int n_lpart = (nb + 255) / 256;
  float* wpart = lpart + n_lpart;
  const int gparts = 2 * n_sms;
  auto grid_for = [&](long long n) { return (int)std::min<long long>((n + 255) / 256, (long long)n_sms * 16); };
  U8Input x{t.images, t.pitch, (size_t)t.pitch * H, H, W};
  F32Input in1{a1, kC, H1, W1}, in2{a2, kC, H2, W2};
  conv_fwd_kernel<1, 2, U8Input><<<grid_for((long long)B * H1 * W1), 256, 0, s>>>(x, t.theta, kOffW1, kOffB1, t.bf16,
                                                                                 t.bf16, a1, B, H1, W1);
  conv_fwd_kernel<kC, 2, F32Input><<<grid_for((long long)B * H2 * W2), 256, 0, s>>>(in1, t.theta, kOffW2, kOffB2,
                                                                                    t.bf16, t.bf16, a2, B, H2, W2);
  conv_fwd_kernel<kC, 1, F32Input><<<grid_for((long long)B * H2 * W2), 256, 0, s>>>(in2, t.theta, kOffW3, kOffB3,
                                                                                    t.bf16, 0, a3, B, H2, W2);
  pool_head_kernel<<<n_lpart, 256, 0, s>>>(a3, B, H2, W2, Th, Tw, t.theta, t.bf16, t.labels, P, z, dz, lpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (t.logits_out) {
    if ((e = cudaMemcpyAsync(t.logits_out, z, sizeof(float) * nb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
  }
  if (!t.labels) return cudaSuccess;  // forward only
  float* grad = t.grad;
  head_grad_kernel<<<kC + 1, 256, 0, s>>>(P, dz, nb, grad, lpart, n_lpart, t.loss);
  dz3_kernel<<<grid_for((long long)na2), 256, 0, s>>>(a3, dz, t.theta, t.bf16, B, H2, W2, Th, Tw, dz3);
  conv_wgrad_kernel<kC, 1, F32Input><<<gparts, 256, 0, s>>>(in2, dz3, B, H2, W2, wpart);
  reduce_parts_kernel<<<(kC * kC * 9 + kC + 255) / 256, 256, 0, s>>>(wpart, gparts, kC * kC * 9, grad, kOffW3, kOffB3);
  conv_dgrad_kernel<1><<<grid_for((long long)B * H2 * W2), 256, 0, s>>>(dz3, H2, W2, a2, H2, W2, t.theta, kOffW3,
                                                                        t.bf16, B, dz2);
  conv_wgrad_kernel<kC, 2, F32Input><<<gparts, 256, 0, s>>>(in1, dz2, B, H2, W2, wpart);
  reduce_parts_kernel<<<(kC * kC * 9 + kC + 255) / 256, 256, 0, s>>>(wpart, gparts, kC * kC * 9, grad, kOffW2, kOffB2);
  conv_dgrad_kernel<2><<<grid_for((long long)B * H1 * W1), 256, 0, s>>>(dz2, H2, W2, a1, H1, W1, t.theta, kOffW2,
                                                                        t.bf16, B, dz1);
  conv_wgrad_kernel<1, 2, U8Input><<<gparts, 256, 0, s>>>(x, dz1, B, H1, W1, wpart);
  reduce_parts_kernel<<<1, 256, 0, s>>>(wpart, gparts, kC * 9, grad, kOffW1, kOffB1);
  if (t.lr > 0.0f) {
    const double b1 = 0.9, b2 = 0.999;
    adam_kernel<<<(kPropParams + 255) / 256, 256, 0, s>>>(t.theta, t.adam_m, t.adam_v, grad, kPropParams, t.lr,
                                                          (float)b1, (float)b2,
                                                          (float)(1.0 - std::pow(b1, (double)t.step)),
                                                          (float)(1.0 - std::pow(b2, (double)t.step)), 1e-8f);
  }
  return cudaGetLastError();
}

}  // namespace cdvs
