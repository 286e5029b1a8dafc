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
//     L = [y^2 | y] W + c, with W = [-1/(2v); mu/v] (64 x 512), on tcgen05
//     with the accumulators in tensor memory;
//   * per image, S = Gamma^T [1 | y | y^2] (512 x 65), from which
//     g_mu = (S_y - mu S_1) / s and g_sigma = (S_yy - 2 mu S_y + mu^2 S_1) / v - S_1,
//     also on tcgen05, its operands written ready by the posterior kernel.
// (The PCA projection, 1/8 of Eq. 10's products, runs on mma.sync inside the
// posterior kernel, whose shared memory holds no room for its operands.)
// Both split their operands into two FP16 halves (x = hi + lo) and take
// three products per term (hi hi + hi lo + lo hi), accumulated in FP32:
// about 22 significant bits per product, so the softmax, which needs the
// log-likelihood to ~1e-5 absolute, stays within FP32-level error.  The
// model's 1/v can be large, so each component's column of W is scaled by a
// power of two into FP16's range on the host and the scale is undone, exactly,
// on the accumulator.  The softmax and every reduction run in a fixed order.
#include <algorithm>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kComp = kScfvComp, kDim = kScfvDim, kIn = 128;

// ---- FP16-split tensor-core products

// (x0, x1) = hi + lo, both halves FP16 pairs (round to nearest)
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 f = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - f.x, x1 - f.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// D = A B + D for one 16 x 8 x 16 block (mma.sync m16n8k16, FP16 in, FP32 accumulate)
__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 16-byte asynchronous copy global -> shared (both 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---- tcgen05: shared-memory matrix descriptors, tensor memory, mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// No-swizzle K-major operand at shared address `a`: 8 x 16-byte core
// matrices, adjacent along K at `lbo` bytes, along M / N at `sbo` bytes.
__device__ __forceinline__ uint64_t tc_desc(uint32_t a, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((a >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version (fixed 0b001); base offset 0, no swizzle
  return d;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Waits for phase `parity` of the mbarrier to complete: at most 2^22 polls
// and 0.2 s (the global nanosecond timer); false when it gave up.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > 200000000ull) return false;
  }
  return false;
}

// 32 consecutive accumulator columns of this warp's 32 lanes (one record per
// lane), read as FP32
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(r[e]);
}

// K_a + K_b: projection and posteriors, persistent CTAs of 8 warps (one per
// SM: the log-likelihoods of a tile fill the SM's 512 tensor-memory
// columns); a tile is 128 records.
//   1. y = (x - m) P^T: warp w takes records 16 (w % 8) .. + 15 and the
//      outputs of its kProjTiles 8-column tiles, FP16 hi / lo operands on
//      mma.sync m16n8k16, three products per term.  y goes to shared memory
//      and to Y.
//   2. The log-likelihoods L = [y^2 | y] W + c on tcgen05: A = [y^2 | y]
//      (128 x 64) split into FP16 halves in shared memory, B = the model's
//      column-scaled W in FP16 halves (staged once per CTA), three products
//      (lo hi, hi lo, hi hi) per half of the 512 components (M = 128,
//      N = 256, K = 16 each), issued by one thread, accumulated in FP32 in
//      tensor memory; one commit to an mbarrier.
//   3. Per record the softmax over the 512 components, read back with
//      tcgen05.ld: warp w reads lanes 32 (w % 4) .. (its records) and
//      components kPartCols (w / 4) .. ; l = acc / e_i + c_i; a running maximum
//      and sum of exponentials, then the posteriors: two passes over the
//      accumulators, the four parts of a record combined in a fixed order.
// Should a tile's products not complete within the bounded wait, the CTA
// sets kStatusTimeout in *status, stops, waits (bounded again) for the
// products still in flight and frees its tensor memory; the gradient kernel
// then writes NaN gradients.  skip_products (a testing hook) leaves the
// products unissued, so that the wait runs out with nothing in flight.
// Fragment layouts of m16n8k16 (f16): lane = 4 g + t; A register q holds
// row g + 8 (q & 1), columns 2t + 8 (q >> 1) + {0, 1}; B register q holds
// rows 2t + 8 q + {0, 1}, column g; C elements (g, 2t), (g, 2t + 1),
// (g + 8, 2t), (g + 8, 2t + 1).
// The posterior kernel's output is the gradient products' operands, laid
// out as the gradient kernel stages them: per chunk of 32 consecutive
// records of the batch (kChunkBytes, 16-byte aligned),
//   Gamma^T hi | Gamma^T lo   MN-major: element (component m, record k) at
//                             (k / 8) 8 KB + (m / 8) 128 + (k % 8) 16 + (m % 8) 2
//   Z hi | Z lo               K-major, Z = [1 | y | y^2 | 0] (80 columns):
//                             element (column n, record k) at
//                             (n / 8) 512 + (k / 8) 128 + (n % 8) 16 + (k % 8) 2
// in FP16 halves (x = hi + lo).  Records past the batch's last are zero.
constexpr int kChunk = 32, kZCols = 80;
constexpr int kGKst = kComp / 8 * 128;                   // 8 KB: Gamma^T bytes between 8-record groups
constexpr int kGBytes = kChunk / 8 * kGKst;              // 32 KB per half
constexpr int kZSbo = kChunk / 8 * 128;                  // 512: Z bytes between 8-column groups
constexpr int kZBytes = kZCols / 8 * kZSbo;              // 5 KB per half
constexpr int kChunkBytes = 2 * kGBytes + 2 * kZBytes;   // 75776
constexpr int kPostTile = 128, kPostThreads = 256, kYPitch = 36;
static_assert(kPostTile % kChunk == 0, "posterior tiles hold whole chunks");
constexpr int kPostWarps = kPostThreads / 32;
constexpr int kPostParts = kPostWarps / 4;          // column parts of a record in the softmax
constexpr int kPartCols = kComp / kPostParts;
constexpr int kProjTiles = 4 / (kPostWarps / 8);    // projection n-tiles per warp
static_assert(kPostWarps == 8 || kPostWarps == 16, "8 or 16 warps");
constexpr int kTcSbo = (2 * kDim / 8) * 128;          // 1024: bytes between 8-row groups of A and B
constexpr int kTcABytes = kPostTile / 8 * kTcSbo;     // 16 KB per half
constexpr int kTcBBytes = kComp / 8 * kTcSbo;         // 64 KB per half
constexpr int kPfWords = 2048;                        // projection fragments per half
// kind::f16 instruction descriptor: FP32 accumulator, FP16 A and B, both K-major, N = 256, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr int kTmemCols = 512;
constexpr float kLog2e = 1.4426950408889634f;
// dynamic shared memory: B hi | B lo | A hi | A lo | projection fragments hi, lo
constexpr int kPostSmemBytes = 2 * kTcBBytes + 2 * kTcABytes + 2 * kPfWords * 4;
static_assert(kScfvWHalfWords * 4 == kTcBBytes, "the model's B halves are the staged ones");

__global__ void __launch_bounds__(kPostThreads, 1) scfv_post_kernel(const float* desc, int n_rec,
                                                                    const float* model, unsigned char* ops,
                                                                    int* status, int skip_products) {
  extern __shared__ __align__(128) unsigned char smb[];
  unsigned char* const Bs = smb;                                 // B hi, then B lo
  unsigned char* const As = smb + 2 * kTcBBytes;                 // A hi, then A lo
  uint32_t* const Pf = reinterpret_cast<uint32_t*>(As + 2 * kTcABytes);
  __shared__ float ys[kPostTile][kYPitch];
  __shared__ __align__(16) float cs[kComp];
  __shared__ __align__(16) float inve[kComp];
  __shared__ float mean[kIn];
  __shared__ float redm[kPostParts][kPostTile], reds[kPostParts][kPostTile];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  if (blockIdx.x * kPostTile >= n_rec) return;
  // the model's operands, 16-byte asynchronous copies all in flight at once
  for (int i = tid; i < 2 * kTcBBytes / 16; i += kPostThreads)
    cp_async16(Bs + 16 * i, reinterpret_cast<const unsigned char*>(model + kScfvOffW) + 16 * i);
  for (int i = tid; i < 2 * kPfWords / 4; i += kPostThreads)
    cp_async16(Pf + 4 * i, reinterpret_cast<const uint32_t*>(model + kScfvOffPf) + 4 * i);
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
  for (int i = tid; i < kComp; i += kPostThreads) {
    cs[i] = model[kScfvOffC + i];
    inve[i] = model[kScfvOffInvE + i];
  }
  for (int i = tid; i < kIn; i += kPostThreads) mean[i] = model[kScfvOffMean + i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B is read by the tensor cores
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  bool inflight = false;  // products of an abandoned tile may still be running
  for (int r0 = blockIdx.x * kPostTile; r0 < n_rec; r0 += gridDim.x * kPostTile) {
    {  // 1. projection: warp w takes records 16 (w % 8) .. + 15 and kProjTiles 8-column output tiles
      const int rw = 16 * (warp & 7), j0 = kProjTiles * (warp >> 3);
      float pa[kProjTiles][4];
#pragma unroll
      for (int j = 0; j < kProjTiles; ++j) pa[j][0] = pa[j][1] = pa[j][2] = pa[j][3] = 0.0f;
      // rows past the last record repeat it (finite values, never stored)
      const float* xa = desc + (size_t)min(r0 + rw + g, n_rec - 1) * kIn;
      const float* xb = desc + (size_t)min(r0 + rw + g + 8, n_rec - 1) * kIn;
      // the loads of four k-steps are issued before any of them is used
#pragma unroll 1
      for (int s0 = 0; s0 < kIn / 16; s0 += 4) {
        float2 v[4][4];
#pragma unroll
        for (int sb = 0; sb < 4; ++sb)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            v[sb][q] = __ldg(reinterpret_cast<const float2*>(((q & 1) ? xb : xa) + 16 * (s0 + sb) + 2 * t + 8 * (q >> 1)));
#pragma unroll
        for (int sb = 0; sb < 4; ++sb) {
          const int s = s0 + sb;
          uint32_t ah[4], al[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 16 * s + 2 * t + 8 * (q >> 1);
            split_h2(v[sb][q].x - mean[c], v[sb][q].y - mean[c + 1], ah[q], al[q]);
          }
#pragma unroll
          for (int j = 0; j < kProjTiles; ++j) {
            const int f = ((s * 4 + j0 + j) * 32 + lane) * 2;
            const uint32_t bh[2] = {Pf[f], Pf[f + 1]}, bl[2] = {Pf[kPfWords + f], Pf[kPfWords + f + 1]};
            mma_f16(pa[j], al, bh);
            mma_f16(pa[j], ah, bl);
            mma_f16(pa[j], ah, bh);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kProjTiles; ++j) {
        const int r = rw + g, c = 8 * (j0 + j) + 2 * t;
        ys[r][c] = pa[j][0];
        ys[r][c + 1] = pa[j][1];
        ys[r + 8][c] = pa[j][2];
        ys[r + 8][c + 1] = pa[j][3];
      }
    }
    __syncthreads();  // ys complete; the previous tile's accumulator reads are done (fenced)
    // Z = [1 | y | y^2 | 0] of the tile's chunks: a 16-byte row per (column
    // n, 8 records) and half; records past the last are zero
    const int n_chunks = (n_rec + kChunk - 1) / kChunk;
    for (int e = tid; e < (kPostTile / 8) * kZCols; e += kPostThreads) {
      const int n = e % kZCols, rg = e / kZCols;  // rg: 8-record group of the tile
      const int C = (r0 + 8 * rg) / kChunk;
      if (C >= n_chunks) continue;
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float z[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int rl = 8 * rg + 2 * u + h;
          float x = 0.0f;
          if (r0 + rl < n_rec) {
            if (n == 0) x = 1.0f;
            else if (n <= kDim) x = ys[rl][n - 1];
            else if (n <= 2 * kDim) x = ys[rl][n - 1 - kDim] * ys[rl][n - 1 - kDim];
          }
          z[h] = x;
        }
        split_h2(z[0], z[1], hi[u], lo[u]);
      }
      unsigned char* zb = ops + (size_t)C * kChunkBytes + 2 * kGBytes;
      const int off = (n >> 3) * kZSbo + (((r0 + 8 * rg) % kChunk) >> 3) * 128 + (n & 7) * 16;
      *reinterpret_cast<uint4*>(zb + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(zb + kZBytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    // A = [y^2 | y] in FP16 halves: 8-element pieces (record r, columns 8 kc ..)
    for (int e = tid; e < kPostTile * 8; e += kPostThreads) {
      const int r = e & (kPostTile - 1), kc = e / kPostTile;
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float y0 = ys[r][8 * (kc & 3) + 2 * u], y1 = ys[r][8 * (kc & 3) + 2 * u + 1];
        if (kc < 4) {
          y0 *= y0;
          y1 *= y1;
        }
        split_h2(y0, y1, hi[u], lo[u]);
      }
      const int off = (r >> 3) * kTcSbo + kc * 128 + (r & 7) * 16;
      *reinterpret_cast<uint4*>(As + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(As + kTcABytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 2. the products, one thread
    if (tid == 0 && !skip_products) {
      tc_fence_after();
      const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int p = 0; p < 3; ++p) {  // lo hi, hi lo, hi hi
          const uint32_t ap = a0 + (p == 0 ? kTcABytes : 0), bp = b0 + (p == 1 ? kTcBBytes : 0) + h * 32 * kTcSbo;
#pragma unroll
          for (int ks = 0; ks < 2 * kDim / 16; ++ks) {
            const uint64_t da = tc_desc(ap + ks * 256, 128, kTcSbo), db = tc_desc(bp + ks * 256, 128, kTcSbo);
            const uint32_t acc = (p | ks) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)(256 * h)),
                "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc));
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&mbar))
                   : "memory");
    }
    // 3. softmax: warp w reads the lanes of quadrant w % 4 (its records) and
    // components kPartCols (w / 4) .., in 32-column pieces.  Pass 1
    // keeps a running maximum m and sum of exp(l - m), rescaled once per
    // piece; the four parts of a record combine in a fixed order.
    const bool ok = mbar_wait(&mbar, phase);
    if (__syncthreads_or(!ok)) {  // uniform: any thread that gave up stops the CTA
      if (tid == 0) atomicOr(status, kStatusTimeout);
      inflight = !skip_products;
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    const int quad = warp & 3, part = warp >> 2, r = 32 * quad + lane, n0 = kPartCols * part;
    const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)n0;
    float m = -3.0e38f, sum = 0.0f;
#pragma unroll 1
    for (int c = 0; c < kPartCols / 32; ++c) {
      float v[32];
      tmem_ld32(taddr + 32 * c, v);
      float cm = -3.0e38f;
#pragma unroll
      for (int e = 0; e < 32; e += 4) {
        const float4 iv = *reinterpret_cast<const float4*>(inve + n0 + 32 * c + e);
        const float4 cv = *reinterpret_cast<const float4*>(cs + n0 + 32 * c + e);
        v[e] = fmaf(v[e], iv.x, cv.x);
        v[e + 1] = fmaf(v[e + 1], iv.y, cv.y);
        v[e + 2] = fmaf(v[e + 2], iv.z, cv.z);
        v[e + 3] = fmaf(v[e + 3], iv.w, cv.w);
        cm = fmaxf(fmaxf(cm, fmaxf(v[e], v[e + 1])), fmaxf(v[e + 2], v[e + 3]));
      }
      const float mn = fmaxf(m, cm), mref = mn * kLog2e;
      float ps = 0.0f;
#pragma unroll
      for (int e = 0; e < 32; ++e) ps += ex2_approx(fmaf(v[e], kLog2e, -mref));
      sum = fmaf(sum, ex2_approx((m - mn) * kLog2e), ps);
      m = mn;
    }
    redm[part][r] = m;
    reds[part][r] = sum;
    __syncthreads();
    float M = redm[0][r];
#pragma unroll
    for (int p = 1; p < kPostParts; ++p) M = fmaxf(M, redm[p][r]);
    float S = 0.0f;
#pragma unroll
    for (int p = 0; p < kPostParts; ++p) S = fmaf(reds[p][r], ex2_approx((redm[p][r] - M) * kLog2e), S);
    const float inv = 1.0f / S;
    const float mref = M * kLog2e;
    // every lane reads (the loads are warp-collective).  A lane's record k of
    // chunk C: 8 components at a time into 16-byte rows of Gamma^T hi / lo;
    // records past the last are written as zero up to the chunk's end.
    const bool live = r0 + r < n_rec;
    const bool in_chunks = r0 + r < kChunk * ((n_rec + kChunk - 1) / kChunk);
    unsigned char* const gb = ops + (size_t)((r0 + r) / kChunk) * kChunkBytes +
                              (((r0 + r) % kChunk) >> 3) * kGKst + ((r0 + r) & 7) * 16;
#pragma unroll 1
    for (int c = 0; c < kPartCols / 32; ++c) {
      float v[32];
      tmem_ld32(taddr + 32 * c, v);
#pragma unroll
      for (int e = 0; e < 32; e += 8) {
        float o[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          o[u] = live ? ex2_approx(fmaf(fmaf(v[e + u], inve[n0 + 32 * c + e + u], cs[n0 + 32 * c + e + u]), kLog2e,
                                        -mref)) * inv
                      : 0.0f;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) split_h2(o[2 * u], o[2 * u + 1], hi[u], lo[u]);
        const int m = n0 + 32 * c + e;  // 8-component group
        if (in_chunks) {
          *reinterpret_cast<uint4*>(gb + (m >> 3) * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(gb + kGBytes + (m >> 3) * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    }
    tc_fence_before();  // these reads precede the next tile's products
  }
  // the abandoned tile's products finish (bounded) before their tensor memory is freed
  if (inflight) mbar_wait(&mbar, phase);
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// K_c: Fisher gradients as per-image products S = Gamma^T [1 | y | y^2]
// (512 x 65, padded to 80 columns) on tcgen05, one CTA of 16 warps per image;
// g_mu = (S_y - mu S_1) / s and g_sigma = (S_yy - 2 mu S_y + mu^2 S_1) / v - S_1.
// The operands come ready from the posterior kernel, chunk by chunk (32
// records of the batch, kChunkBytes): one bulk asynchronous copy stages a
// chunk into one of two operand buffers, completing on that buffer's
// mbarrier.  In the image's first and last chunk the records of the
// neighbouring images keep their posteriors but get zero rows of Z, so they
// add nothing.  Per chunk one thread issues 24 products (four 128-component
// blocks x two k-steps x lo hi, hi lo, hi hi; M = 128, N = 80, K = 16) into
// 4 x 80 tensor-memory columns, accumulated over the image's chunks; once a
// chunk's products complete, its buffer takes the chunk two ahead.  Then
// warp w reads the accumulators of component block w / 4, lanes of quadrant
// w % 4: thread = component, its 65 sums in registers, and writes its row
// of g_mu and g_sigma.  Every wait is bounded.
constexpr int kGradThreads = 512;
// kind::f16: FP32 accumulator, FP16 A (MN-major) and B (K-major), N = 80, M = 128
constexpr uint32_t kGradIdesc =
    (1u << 4) | (1u << 15) | ((uint32_t)(kZCols >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr int kGradSmemBytes = 2 * kChunkBytes;

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, int bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// One thread: the 24 products of the chunk in buffer `buf`, then a commit to
// `bar`.  da0 / db0 describe buffer 0's Gamma^T hi and Z hi; every other
// operand differs in its start address only (the low field, 16-byte units;
// shared addresses stay below 256 KB, so the sum never carries out).
__device__ __forceinline__ void grad_issue(uint32_t tmem, uint64_t da0, uint64_t db0, int buf, bool first,
                                           uint64_t* bar) {
  tc_fence_after();
  const uint64_t b16 = (uint64_t)(buf * kChunkBytes) >> 4;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int p = 0; p < 3; ++p) {  // lo hi, hi lo, hi hi
#pragma unroll
      for (int ks = 0; ks < kChunk / 16; ++ks) {
        const uint64_t da = da0 + b16 + (uint64_t)(((p == 0 ? kGBytes : 0) + j * 2048 + ks * 2 * kGKst) >> 4);
        const uint64_t db = db0 + b16 + (uint64_t)(((p == 1 ? kZBytes : 0) + ks * 256) >> 4);
        const uint32_t acc = (first && p == 0 && ks == 0) ? 0u : 1u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)(kZCols * j)),
            "l"(da), "l"(db), "r"(kGradIdesc), "r"(acc));
      }
    }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__global__ void __launch_bounds__(kGradThreads, 1) scfv_grad_kernel(const unsigned char* ops, const int* rec_off,
                                                                    const float* model, float* g_mu, float* g_sig,
                                                                    int* status) {
  extern __shared__ __align__(128) unsigned char gsm[];
  __shared__ __align__(8) uint64_t bars[4];  // copies into buffer 0, 1; products from buffer 0, 1
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float nan = __int_as_float(0x7fc00000);
  const int t0 = rec_off[b], t1 = rec_off[b + 1];
  if ((*status & kStatusTimeout) || t1 <= t0) {
    // incomplete posteriors: NaN; no descriptor: zero gradients
    const float v = t1 <= t0 && !(*status & kStatusTimeout) ? 0.0f : nan;
    for (int e = tid; e < kComp * kDim; e += kGradThreads) {
      g_mu[(size_t)b * kComp * kDim + e] = v;
      g_sig[(size_t)b * kComp * kDim + e] = v;
    }
    return;
  }
  const int C0 = t0 / kChunk, n_ch = (t1 - 1) / kChunk - C0 + 1;
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[q])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
    for (int q = 0; q < 2 && q < n_ch; ++q)  // chunks 0 and 1 on their way
      bulk_copy(gsm + q * kChunkBytes, ops + (size_t)(C0 + q) * kChunkBytes, kChunkBytes, &bars[q]);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint64_t da0 = tc_desc(smem_addr(gsm), kGKst, 128);               // MN-major: K stride, M stride
  const uint64_t db0 = tc_desc(smem_addr(gsm + 2 * kGBytes), 128, kZSbo);  // K-major
  uint32_t cph[2] = {0u, 0u};  // parity of each buffer's next copy completion
  uint32_t mph[2] = {0u, 0u};  // (thread 0) parity of each buffer's next product completion
  bool copy_out[2] = {n_ch > 0, n_ch > 1};  // (thread 0) copies issued, not yet seen complete by all
  bool failed = false;
  int last_issued = -1;  // the last chunk whose products were issued
  for (int c = 0; c < n_ch; ++c) {
    const int s = c & 1;
    unsigned char* const buf = gsm + s * kChunkBytes;
    const bool ok = mbar_wait(&bars[s], cph[s]);  // chunk c staged
    if (__syncthreads_or(!ok || abort_flag)) {
      failed = true;
      break;
    }
    cph[s] ^= 1u;
    copy_out[s] = false;
    // records of the chunk outside the image: zero Z rows (both halves)
    const int g0 = (C0 + c) * kChunk;
    const int lo = max(t0 - g0, 0), hi = min(t1 - g0, kChunk);
    if (lo > 0 || hi < kChunk) {
      for (int e = tid; e < kChunk * kZCols; e += kGradThreads) {
        const int k = e / kZCols, n = e - k * kZCols;
        if (k >= lo && k < hi) continue;
        const int off = 2 * kGBytes + (n >> 3) * kZSbo + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
        *reinterpret_cast<__half*>(buf + off) = __float2half_rn(0.0f);
        *reinterpret_cast<__half*>(buf + kZBytes + off) = __float2half_rn(0.0f);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // read by the tensor cores
      __syncthreads();
    }
    last_issued = c;
    if (tid == 0) {
      grad_issue(tmem, da0, db0, s, c == 0, &bars[2 + s]);
      if (c + 2 < n_ch) {  // this buffer takes chunk c + 2 once the products have read it
        if (mbar_wait(&bars[2 + s], mph[s])) {
          mph[s] ^= 1u;
          bulk_copy(buf, ops + (size_t)(C0 + c + 2) * kChunkBytes, kChunkBytes, &bars[s]);
          copy_out[s] = true;
        } else {
          abort_flag = 1;
        }
      }
    }
  }
  // every product complete before the accumulators are read or freed: the
  // last issued chunk's commit covers all earlier products.  Its buffer's
  // barrier completes once per chunk of that parity, so the wait is for
  // phase last_issued / 2; the earlier phases are complete (the chunk was
  // staged only after them), so the parity is unambiguous.
  if (last_issued >= 0 && !mbar_wait(&bars[2 + (last_issued & 1)], (uint32_t)((last_issued >> 1) & 1)))
    failed = true;
  // (thread 0) copies still in flight land before the kernel ends
  if (tid == 0)
    for (int q = 0; q < 2; ++q)
      if (copy_out[q] && !mbar_wait(&bars[q], cph[q])) failed = true;
  failed = __syncthreads_or(failed);
  tc_fence_after();
  if (failed) {
    if (tid == 0) atomicOr(status, kStatusTimeout);
    for (int e = tid; e < kComp * kDim; e += kGradThreads) {
      g_mu[(size_t)b * kComp * kDim + e] = nan;
      g_sig[(size_t)b * kComp * kDim + e] = nan;
    }
  } else {
    // thread = component i: S_1, S_y, S_yy from its accumulator lane
    const int j = warp >> 2, quad = warp & 3, i = 128 * j + 32 * quad + lane;
    const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(kZCols * j);
    float sa[32], sb[32], s0;
    {
      float v[32];
      tmem_ld32(taddr, v);  // columns 0 .. 31: S_1, S_y[0 .. 30]
      s0 = v[0];
#pragma unroll
      for (int k = 0; k < 31; ++k) sa[k] = v[k + 1];
      tmem_ld32(taddr + 32, v);  // columns 32 .. 63: S_y[31], S_yy[0 .. 30]
      sa[31] = v[0];
#pragma unroll
      for (int k = 0; k < 31; ++k) sb[k] = v[k + 1];
      tmem_ld32(taddr + 64, v);  // columns 64 ..: S_yy[31]
      sb[31] = v[0];
    }
    const float inv = 1.0f / (float)(t1 - t0);
    const float nm = inv * model[kScfvOffNmu + i], ns = inv * model[kScfvOffNsig + i];
    // the component's mu and 1/s rows (128-byte aligned) as 16-byte loads
    const float4* mu4 = reinterpret_cast<const float4*>(model + kScfvOffMu + (size_t)i * kDim);
    const float4* isd4 = reinterpret_cast<const float4*>(model + kScfvOffIsd + (size_t)i * kDim);
    // rows of g_mu and g_sigma into the (now idle) operand buffers, 36-float
    // pitch, then out by coalesced 16-byte stores
    constexpr int kRowP = 36;
    float4* om = reinterpret_cast<float4*>(reinterpret_cast<float*>(gsm) + (size_t)i * kRowP);
    float4* os = reinterpret_cast<float4*>(reinterpret_cast<float*>(gsm) + (size_t)(kComp + i) * kRowP);
#pragma unroll
    for (int k4 = 0; k4 < kDim / 4; ++k4) {
      const float4 m4 = __ldg(mu4 + k4), d4 = __ldg(isd4 + k4);
      const float mv[4] = {m4.x, m4.y, m4.z, m4.w}, dv[4] = {d4.x, d4.y, d4.z, d4.w};
      float gm[4], gs[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = 4 * k4 + u;
        const float m = mv[u], d = dv[u];
        gm[u] = nm * d * fmaf(-m, s0, sa[k]);
        gs[u] = ns * fmaf(d * d, fmaf(m, fmaf(m, s0, -2.0f * sa[k]), sb[k]), -s0);
      }
      om[k4] = make_float4(gm[0], gm[1], gm[2], gm[3]);
      os[k4] = make_float4(gs[0], gs[1], gs[2], gs[3]);
    }
    __syncthreads();
    const float4* sm4 = reinterpret_cast<const float4*>(gsm);
    float4* gm4 = reinterpret_cast<float4*>(g_mu + (size_t)b * kComp * kDim);
    float4* gs4 = reinterpret_cast<float4*>(g_sig + (size_t)b * kComp * kDim);
    for (int e = tid; e < kComp * kDim / 4; e += kGradThreads) {
      const int row = e / (kDim / 4), c4 = e - row * (kDim / 4);
      gm4[e] = sm4[row * (kRowP / 4) + c4];
      gs4[e] = sm4[(kComp + row) * (kRowP / 4) + c4];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
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

size_t scfv_ops_bytes(int n_rec) { return (size_t)((n_rec + kChunk - 1) / kChunk) * kChunkBytes; }

cudaError_t launch_scfv(const float* desc, int n_rec, const int* rec_off, int n_images, const float* model,
                        int n_select, void* ops, float* g_mu, float* g_sig, float* delta, int* order,
                        uint32_t* bits, int* status, int skip_products, int n_sms, cudaStream_t s) {
  if (n_images <= 0) return cudaSuccess;
  if (n_rec > 0) {
    const int pbytes = kPostSmemBytes;
    static LaunchCache post_cache;
    cudaError_t e = prepare_launch(scfv_post_kernel, post_cache, pbytes, kPostThreads, nullptr);
    if (e != cudaSuccess) return e;
    scfv_post_kernel<<<std::max(1, std::min((n_rec + kPostTile - 1) / kPostTile, n_sms)), kPostThreads, pbytes, s>>>(
        desc, n_rec, model, static_cast<unsigned char*>(ops), status, skip_products);
  }
  const int gbytes = kGradSmemBytes;
  static LaunchCache grad_cache;
  cudaError_t e = prepare_launch(scfv_grad_kernel, grad_cache, gbytes, kGradThreads, nullptr);
  if (e != cudaSuccess) return e;
  scfv_grad_kernel<<<n_images, kGradThreads, gbytes, s>>>(static_cast<const unsigned char*>(ops), rec_off, model,
                                                          g_mu, g_sig, status);
  scfv_rank_kernel<<<n_images, kComp, 0, s>>>(g_mu, n_select, delta, order, bits);
  return cudaGetLastError();
}

}  // namespace cdvs
