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
// and the sign bits of g_mu for the first n_select of them.
//
// The two contractions run on the tensor cores, as the paper's matrix form
// has them (Eq. 10, 12, 14):
//   * the log-likelihoods of a tile of records against all 512 components,
//     L = [y^2 | y] W + c, with W = [-1/(2v); mu/v] (64 x 512);
//   * per image, S = Gamma^T [1 | y | y^2] (512 x 65), from which
//     g_mu = (S_y - mu S_1) / s and g_sigma = (S_yy - 2 mu S_y + mu^2 S_1) / v - S_1.
// Both split their operands in two (x = hi + lo) and take three products per
// term (hi hi + hi lo + lo hi), accumulated in FP32: about 21 significant
// bits per product, so the softmax, which needs the log-likelihood to ~1e-5
// absolute, stays within FP32-level error.  The log-likelihoods use TF32
// halves (mma.sync m16n8k8: the model's 1/v can be large, and TF32 keeps
// FP32's range); the gradient products use FP16 halves (m16n8k16, twice the
// rate; every operand there is bounded).  The softmax and every reduction
// run in a fixed order.
#include <algorithm>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kComp = kScfvComp, kDim = kScfvDim, kIn = 128;

// ---- split-TF32 tensor-core products

// x = hi + lo with hi, lo both representable in TF32 (round to nearest).
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
  const float r = x - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

// D = A B + D for one 16 x 8 x 8 block (A row-major 16 x 8, B 8 x 8).
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// hi*hi + hi*lo + lo*hi, the small products first
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// K_a + K_b: projection and posteriors.  Persistent CTAs of 8 warps; a tile
// is 64 records (four 16-row tensor-core tiles).
//   1. y = (x - m) P^T on the tensor cores: the tile's descriptors minus the
//      PCA mean (FP32) times P^T (staged once per CTA, split into TF32
//      hi / lo); warp w computes the 16 x 8 output blocks (w / 2, 2 (w % 2))
//      and (w / 2, 2 (w % 2) + 1).  y goes to shared memory and to Y.
//   2. the log-likelihoods L = [y^2 | y] W + c: warp w owns components
//      64w .. 64w + 63 (eight 8-column tiles) for all four row tiles; W is
//      staged once per CTA in fragment order.
//   3. per record the softmax over the 512 components, in a fixed order.
// The fragment layouts of m16n8k8: lane = 4 g + t; A element
// (g + 8 (q & 1), t + 4 (q >> 1)) in register q; B elements (t, g) and
// (t + 4, g); C elements (g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1).
constexpr int kPostTile = 64, kPostThreads = 256, kYPitch = 36, kXPitch = 132;
constexpr float kLog2e = 1.4426950408889634f;

// dynamic shared memory of K_b (floats): W | P^T hi, lo in fragment order |
// the descriptor tile
constexpr int kPostSmemFloats = 2 * kDim * kComp + 2 * kIn * kDim + kPostTile * kXPitch;

__global__ void __launch_bounds__(kPostThreads, 1) scfv_post_kernel(const float* desc, int n_rec,
                                                                    const float* model, float* Y, float* Q) {
  extern __shared__ float4 w4[];
  float* const Ws = reinterpret_cast<float*>(w4);
  uint32_t* const Ph = reinterpret_cast<uint32_t*>(Ws + 2 * kDim * kComp);  // [16 k-steps][4 n-tiles][32 lanes][2]
  uint32_t* const Pl = Ph + kIn * kDim;
  float* const xs = reinterpret_cast<float*>(Pl + kIn * kDim);               // [64][kXPitch]
  __shared__ float ys[kPostTile][kYPitch];
  __shared__ float cs[kComp];
  __shared__ float mean[kIn];
  __shared__ float red[kPostThreads / 32][kPostTile];
  __shared__ float tmax[kPostTile], tinv[kPostTile];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  for (int i = tid; i < 2 * kDim * kComp / 4; i += kPostThreads)
    w4[i] = reinterpret_cast<const float4*>(model + kScfvOffW)[i];
  // P^T (model: pt[k][j], k = input dimension, j = output dimension) in B
  // fragment order for k-step s, n-tile j8: (k = 8s + t (+4), j = 8 j8 + g)
  for (int i = tid; i < kIn * kDim; i += kPostThreads) {
    const int e = i & 1, ln = (i >> 1) & 31, j8 = (i >> 6) & 3, ks = i >> 8;
    const int k = 8 * ks + (ln & 3) + 4 * e, j = 8 * j8 + (ln >> 2);
    split_tf32(model[kScfvOffPcaT + k * kDim + j], Ph[i], Pl[i]);
  }
  for (int i = tid; i < kComp; i += kPostThreads) cs[i] = model[kScfvOffC + i];
  for (int i = tid; i < kIn; i += kPostThreads) mean[i] = model[kScfvOffMean + i];
  const float2* wf = reinterpret_cast<const float2*>(w4) + warp * 8 * 8 * 32;
  for (int r0 = blockIdx.x * kPostTile; r0 < n_rec; r0 += gridDim.x * kPostTile) {
    __syncthreads();  // model staged; the previous tile is done with xs, ys, red, tmax, tinv
    for (int e = tid; e < kPostTile * kIn / 4; e += kPostThreads) {
      const int r = e / (kIn / 4), c4 = e - r * (kIn / 4);
      float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (r0 + r < n_rec) {
        v = reinterpret_cast<const float4*>(desc + (size_t)(r0 + r) * kIn)[c4];
        v.x -= mean[4 * c4];
        v.y -= mean[4 * c4 + 1];
        v.z -= mean[4 * c4 + 2];
        v.w -= mean[4 * c4 + 3];
      }
      *reinterpret_cast<float4*>(xs + r * kXPitch + 4 * c4) = v;
    }
    __syncthreads();
    {  // 1. projection: blocks (mt, nt) and (mt, nt + 1) of the 64 x 32 output
      const int mt = warp >> 1, nt0 = 2 * (warp & 1);
      float pa[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
#pragma unroll 4
      for (int ks = 0; ks < kIn / 8; ++ks) {
        uint32_t ah[4], al[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          split_tf32(xs[(16 * mt + g + 8 * (q & 1)) * kXPitch + 8 * ks + t + 4 * (q >> 1)], ah[q], al[q]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int f = ((ks * 4 + nt0 + u) * 32 + lane) * 2;
          const uint32_t bh[2] = {Ph[f], Ph[f + 1]}, bl[2] = {Pl[f], Pl[f + 1]};
          mma3(pa[u], ah, al, bh, bl);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int r = 16 * mt + g, c = 8 * (nt0 + u) + 2 * t;
        ys[r][c] = pa[u][0];
        ys[r][c + 1] = pa[u][1];
        ys[r + 8][c] = pa[u][2];
        ys[r + 8][c + 1] = pa[u][3];
      }
    }
    __syncthreads();
    for (int e = tid; e < kPostTile * kDim; e += kPostThreads) {
      const int r = e / kDim, k = e - r * kDim;
      if (r0 + r < n_rec) Y[(size_t)(r0 + r) * kDim + k] = ys[r][k];
    }
    // 2. log-likelihoods
    float acc[4][8][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][j][q] = 0.0f;
#pragma unroll 1
    for (int s = 0; s < 8; ++s) {
      // A = [y^2 | y]: k-steps 0..3 take the squares of dimensions 8s..8s+7,
      // k-steps 4..7 the dimensions themselves
      uint32_t ah[4][4], al[4][4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float y = ys[16 * m + g + 8 * (q & 1)][8 * (s & 3) + t + 4 * (q >> 1)];
          split_tf32(s < 4 ? y * y : y, ah[m][q], al[m][q]);
        }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 w = wf[(s * 8 + j) * 32 + lane];
        uint32_t bh[2], bl[2];
        split_tf32(w.x, bh[0], bl[0]);
        split_tf32(w.y, bh[1], bl[1]);
#pragma unroll
        for (int m = 0; m < 4; ++m) mma3(acc[m][j], ah[m], al[m], bh, bl);
      }
    }
    // 3. softmax per record: records 16m + g + 8h of this lane (h = q >> 1),
    // components 64 warp + 8j + 2t + (q & 1)
    float mx[4][2];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v = -3.0e38f;
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            float& l = acc[m][j][2 * h + e];
            l += cs[64 * warp + 8 * j + 2 * t + e];
            v = fmaxf(v, l);
          }
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 2));
        mx[m][h] = v;
      }
    if (t == 0)
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) red[warp][16 * m + g + 8 * h] = mx[m][h];
    __syncthreads();
    if (tid < kPostTile) {
      float v = red[0][tid];
      for (int w = 1; w < kPostThreads / 32; ++w) v = fmaxf(v, red[w][tid]);
      tmax[tid] = v;
    }
    __syncthreads();
    float sm[4][2];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float mref = tmax[16 * m + g + 8 * h] * kLog2e;
        float v = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            float& l = acc[m][j][2 * h + e];
            l = ex2_approx(fmaf(l, kLog2e, -mref));
            v += l;
          }
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        sm[m][h] = v;
      }
    __syncthreads();  // every max read before red is rewritten
    if (t == 0)
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) red[warp][16 * m + g + 8 * h] = sm[m][h];
    __syncthreads();
    if (tid < kPostTile) {
      float v = 0.0f;
      for (int w = 0; w < kPostThreads / 32; ++w) v += red[w][tid];
      tinv[tid] = 1.0f / v;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = 16 * m + g + 8 * h;
        if (r0 + r >= n_rec) continue;
        const float inv = tinv[r];
        float2* out = reinterpret_cast<float2*>(Q + (size_t)(r0 + r) * kComp + 64 * warp + 2 * t);
#pragma unroll
        for (int j = 0; j < 8; ++j) out[4 * j] = make_float2(acc[m][j][2 * h] * inv, acc[m][j][2 * h + 1] * inv);
      }
  }
}

// K_c: Fisher gradients as per-image products S = Gamma^T [1 | y | y^2]
// (512 x 65, padded to 72 columns), one CTA per image: warp w owns
// components 32w .. 32w + 31 (two 16-row tiles) and all nine 8-column tiles.
// The image's records go through in chunks of 32 (two 16-deep k-steps); the
// chunk's posteriors arrive by asynchronous copies, double-buffered, while
// the previous chunk is multiplied.  Operands are split into FP16 hi / lo
// (x = hi + lo, 22 significant bits; posteriors lie in [0, 1] and
// [1 | y | y^2] within +-4 for the projections of unit descriptors on the
// orthonormal PCA rows, far inside FP16's range) and multiplied by
// mma.sync m16n8k16 with FP32 accumulation, three products per term.  The
// [1 | y | y^2] chunk is split once, into shared memory, for all warps.
// Fragment layouts of m16n8k16 (f16): lane = 4 g + t; A register q holds
// row g + 8 (q & 1), columns 2t + 8 (q >> 1) + {0, 1}; B register q holds
// rows 2t + 8 q + {0, 1}, column g; C as for m16n8k8.
constexpr int kGradChunk = 32, kGradThreads = 512, kZCols = 72, kQPitch = kComp + 8, kSPitch = 73;
// dynamic shared memory (32-bit words): two posterior chunks | Z hi, lo as
// record pairs | (after the loop) S for 256 components at a time
constexpr int kGradQWords = kGradChunk * kQPitch;
constexpr int kGradZWords = (kGradChunk / 2) * kZCols;
constexpr int kGradSmemWords = 2 * kGradQWords + 2 * kGradZWords;
static_assert(256 * kSPitch <= 2 * kGradQWords, "S of 256 components fits the posterior buffers");

__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 f = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - f.x, x1 - f.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}

// Posteriors of records c0 .. c0 + nr - 1 (nr <= 32) into a chunk buffer;
// the rows past nr are zeroed.
__device__ __forceinline__ void load_q_chunk(const float* Q, int c0, int nr, float* qs) {
  for (int e = threadIdx.x; e < kGradChunk * kComp / 4; e += kGradThreads) {
    const int r = e / (kComp / 4), c4 = e - r * (kComp / 4);
    float* dst = qs + r * kQPitch + 4 * c4;
    if (r < nr) cp_async16(dst, Q + (size_t)(c0 + r) * kComp + 4 * c4);
    else *reinterpret_cast<float4*>(dst) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(kGradThreads, 1) scfv_grad_kernel(const float* Y, const float* Q, const int* rec_off,
                                                                    const float* model, float* g_mu, float* g_sig) {
  extern __shared__ float4 gsm4[];
  float* const qbuf = reinterpret_cast<float*>(gsm4);                       // 2 x [32][kQPitch]
  uint32_t* const zh = reinterpret_cast<uint32_t*>(qbuf + 2 * kGradQWords);  // [16 record pairs][72]
  uint32_t* const zl = zh + kGradZWords;
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  const int t0 = rec_off[b], t1 = rec_off[b + 1];
  float acc[2][kZCols / 8][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < kZCols / 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[m][j][q] = 0.0f;
  if (t0 < t1) load_q_chunk(Q, t0, min(kGradChunk, t1 - t0), qbuf);
  for (int c0 = t0, buf = 0; c0 < t1; c0 += kGradChunk, buf ^= 1) {
    const int nr = min(kGradChunk, t1 - c0);
    // [1 | y | y^2] of the chunk, split, as record pairs (every warp is past
    // the previous chunk's products: the barrier at the end of the loop)
    for (int e = tid; e < kGradZWords; e += kGradThreads) {
      const int rp = e / kZCols, c = e - rp * kZCols;
      float z[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = 2 * rp + h;
        z[h] = 0.0f;
        if (r < nr) {
          if (c == 0) z[h] = 1.0f;
          else if (c <= kDim) z[h] = Y[(size_t)(c0 + r) * kDim + c - 1];
          else if (c <= 2 * kDim) {
            const float y = Y[(size_t)(c0 + r) * kDim + c - 1 - kDim];
            z[h] = y * y;
          }
        }
      }
      split_h2(z[0], z[1], zh[e], zl[e]);
    }
    // the next chunk's posteriors on their way; this chunk's have landed
    if (c0 + kGradChunk < t1) {
      load_q_chunk(Q, c0 + kGradChunk, min(kGradChunk, t1 - c0 - kGradChunk), qbuf + (buf ^ 1) * kGradQWords);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const float* qs = qbuf + buf * kGradQWords;
#pragma unroll
    for (int s = 0; s < kGradChunk / 16; ++s) {
      // A = Gamma^T: rows = components 32 warp + 16 m .., columns = records 16 s ..
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = 32 * warp + 16 * m + g + 8 * (q & 1);
          const int r = 16 * s + 2 * t + 8 * (q >> 1);
          split_h2(qs[r * kQPitch + c], qs[(r + 1) * kQPitch + c], ah[m][q], al[m][q]);
        }
#pragma unroll
      for (int j = 0; j < kZCols / 8; ++j) {
        const int rp = 8 * s + t, col = 8 * j + g;
        const uint32_t bh[2] = {zh[rp * kZCols + col], zh[(rp + 4) * kZCols + col]};
        const uint32_t bl[2] = {zl[rp * kZCols + col], zl[(rp + 4) * kZCols + col]};
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          mma_f16(acc[m][j], al[m], bh);
          mma_f16(acc[m][j], ah[m], bl);
          mma_f16(acc[m][j], ah[m], bh);
        }
      }
    }
    __syncthreads();  // the chunk's buffers are rewritten next
  }
  // S rows = components, columns = [1 | y | y^2 | pad], 256 components at a
  // time in the posterior buffers, then the gradients
  const int K = t1 - t0;
  const float inv = K > 0 ? 1.0f / (float)K : 0.0f;
  float* const S = qbuf;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    if ((warp >> 3) == half) {
      const int rl = 32 * (warp & 7);
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int j = 0; j < kZCols / 8; ++j) {
          S[(rl + 16 * m + g) * kSPitch + 8 * j + 2 * t] = acc[m][j][0];
          S[(rl + 16 * m + g) * kSPitch + 8 * j + 2 * t + 1] = acc[m][j][1];
          S[(rl + 16 * m + g + 8) * kSPitch + 8 * j + 2 * t] = acc[m][j][2];
          S[(rl + 16 * m + g + 8) * kSPitch + 8 * j + 2 * t + 1] = acc[m][j][3];
        }
    }
    __syncthreads();
    for (int e = tid; e < 256 * kDim; e += kGradThreads) {
      const int il = e / kDim, k = e - il * kDim, i = 256 * half + il;
      const float s0 = S[il * kSPitch], s1 = S[il * kSPitch + 1 + k], s2 = S[il * kSPitch + 1 + kDim + k];
      const float mu = model[kScfvOffMu + i * kDim + k], isd = model[kScfvOffIsd + i * kDim + k];
      const float nm = inv * model[kScfvOffNmu + i], ns = inv * model[kScfvOffNsig + i];
      const size_t o = ((size_t)b * kComp + i) * kDim + k;
      g_mu[o] = nm * isd * fmaf(-mu, s0, s1);
      g_sig[o] = ns * fmaf(isd * isd, fmaf(mu, fmaf(mu, s0, -2.0f * s1), s2), -s0);
    }
    __syncthreads();
  }
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
    const int pbytes = (int)(sizeof(float) * kPostSmemFloats);
    static LaunchCache post_cache;
    cudaError_t e = prepare_launch(scfv_post_kernel, post_cache, pbytes, kPostThreads, nullptr);
    if (e != cudaSuccess) return e;
    scfv_post_kernel<<<std::max(1, std::min((n_rec + kPostTile - 1) / kPostTile, n_sms)), kPostThreads, pbytes, s>>>(
        desc, n_rec, model, Y, Q);
  }
  const int gbytes = (int)(sizeof(float) * kGradSmemWords);
  static LaunchCache grad_cache;
  cudaError_t e = prepare_launch(scfv_grad_kernel, grad_cache, gbytes, kGradThreads, nullptr);
  if (e != cudaSuccess) return e;
  scfv_grad_kernel<<<n_images, kGradThreads, gbytes, s>>>(Y, Q, rec_off, model, g_mu, g_sig);
  scfv_rank_kernel<<<n_images, kComp, 0, s>>>(g_mu, n_select, delta, order, bits);
  return cudaGetLastError();
}

}  // namespace cdvs
