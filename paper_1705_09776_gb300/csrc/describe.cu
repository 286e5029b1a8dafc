// describe.cu -- Alg. 2 on the GPU: dominant orientations (stage A) and
// 128-D descriptors (stage B), then the packing of the (point, orientation)
// records of the whole batch.
//
// One warp per selected point: the warp stages the point's patch of its
// Gaussian level in shared memory (coalesced row loads), builds the 36-bin
// orientation histogram from it, finds the orientations, and for each one
// builds the 4x4x8 descriptor histogram.  The lanes stride over the pixels of
// the sampling disc and add their votes to a per-warp histogram with 32-bit
// integer atomics on a 2^-13 fixed-point scale: integer addition is
// associative, so the sums do not depend on the order in which lanes land.
#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr float kTwoPi = 6.283185307179586f;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }

template <typename StoreT>
struct LevelView {
  const StoreT* base;
  int W, H, pitch;
  __device__ __forceinline__ float at(int x, int y) const { return ld(base + (size_t)y * pitch + x); }
  // central differences, clamp-to-edge
  __device__ __forceinline__ void grad(int u, int v, float& gx, float& gy) const {
    gx = at(min(u + 1, W - 1), v) - at(max(u - 1, 0), v);
    gy = at(u, min(v + 1, H - 1)) - at(u, max(v - 1, 0));
  }
};

__device__ __forceinline__ int desc_level(float so, float sigma0) {
  const int k = (int)roundf((float)(kScales - 1) * log2f(so / sigma0));
  return min(max(k, 0), kScales - 1);
}

template <typename StoreT>
__device__ __forceinline__ LevelView<StoreT> level_of(const DescribeArgs& a, int img, int o, int k) {
  const OctPlan op = a.plans[img].oct[o];
  LevelView<StoreT> v;
  v.base = reinterpret_cast<const StoreT*>(a.levels) + op.level_off + (size_t)k * op.lpitch * op.H;
  v.W = op.W;
  v.H = op.H;
  v.pitch = op.lpitch;
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
  for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Votes are summed as unsigned 32-bit fixed point.  A vote is |g| times
// weights <= 1 with |g| <= 255 * sqrt(2) < 512, so n votes stay below
// 512 n; the scale is the largest power of two <= 2^13 that keeps 512 n
// below 2^32 for the n pixels of the sampling box.  The scaled vote is rounded
// by adding 1.5 * 2^23 in FP32 (exact for values below 2^22) and reading the
// mantissa.
constexpr int kFWarps = 8;

__device__ __forceinline__ float vote_scale(int n_pixels) {
  int sh = 13;
  while (sh > 0 && (512.0 * (double)(n_pixels + 1)) * (double)(1 << sh) >= 4294967296.0) --sh;
  return (float)(1 << sh);
}

__device__ __forceinline__ void vote(unsigned* h, float w, float scale) {
  const unsigned q = (unsigned)(__float_as_int(fmaf(w, scale, 12582912.0f)) - 0x4B400000);
  atomicAdd(h, q);
}

// Walks the bw x bh box starting at (u0, v0): calls f(u, v) for the box
// pixels of this lane (index lane, lane + 32, ...) without a division per step.
template <typename F>
__device__ __forceinline__ void for_box(int u0, int v0, int bw, int bh, int lane, F&& f) {
  if (bw <= 0 || bh <= 0) return;
  const int dq = 32 / bw, dr = 32 - dq * bw;
  int vv = lane / bw, uu = lane - vv * bw;
  for (int i = lane; i < bw * bh; i += 32) {
    f(u0 + uu, v0 + vv);
    uu += dr;
    vv += dq;
    if (uu >= bw) {
      uu -= bw;
      ++vv;
    }
  }
}

// ---- Alg. 2, fused per point.  Stage A: 36-bin histogram of atan2(gy, gx)
// over the disc of radius ori_radius * sigma, weight
// |g| exp(-d^2 / (2 (ori_wsig sigma)^2)); orientations at bins strictly above
// both circular neighbours and above ori_ratio * max, refined by a parabola
// through three bins, in order of bin value.  Stage B, per orientation: 4x4
// cells of side cell_side * sigma in the frame rotated by -theta, 8 bins of
// the gradient angle relative to theta, trilinear votes weighted by
// |g| exp(-(u^2+v^2) / (2 desc_wsig^2)) ((u, v) in cells) over the disc of
// radius desc_radius * sigma; L2-normalise, clamp at 0.2, renormalise.
// Records and descriptors go to per-point staging slots (max_ori each).
template <typename StoreT>
__global__ void __launch_bounds__(kFWarps * 32) describe_kernel(const __grid_constant__ DescribeArgs a) {
  extern __shared__ float4 smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = a.patch_side;
  float* patch = reinterpret_cast<float*>(smem4) + (size_t)warp * P * P;
  unsigned* hist = reinterpret_cast<unsigned*>(reinterpret_cast<float*>(smem4) + (size_t)kFWarps * P * P) +
                   warp * (36 + 128);
  unsigned* ho = hist;        // 36 orientation bins
  unsigned* hd = hist + 36;   // 128 descriptor bins
  const int slot = blockIdx.x * kFWarps + warp;
  if (slot >= a.n_images * a.N) return;
  const int img = slot / a.N, rank = slot - img * a.N;
  if (rank >= a.sel_count[img]) return;
  const Cand c = a.sel[slot];
  const int k = desc_level(c.so, a.sigma0);
  const LevelView<StoreT> G = level_of<StoreT>(a, img, c.octave, k);
  const float Rd = a.desc_radius * c.so, Ro = a.ori_radius * c.so;
  const float R = fmaxf(Rd, a.upright ? 0.0f : Ro);
  const int u0 = max((int)ceilf(c.xo - R), 0), u1 = min((int)floorf(c.xo + R), G.W - 1);
  const int v0 = max((int)ceilf(c.yo - R), 0), v1 = min((int)floorf(c.yo + R), G.H - 1);
  // the patch: the sampling box plus the pixels its gradients read
  const int pu0 = max(u0 - 1, 0), pu1 = min(u1 + 1, G.W - 1);
  const int pv0 = max(v0 - 1, 0), pv1 = min(v1 + 1, G.H - 1);
  const int pw = pu1 - pu0 + 1, ph = pv1 - pv0 + 1;
  const bool staged = pw > 0 && ph > 0 && pw <= P && ph <= P;
  if (staged) {
    for (int r = 0; r < ph; ++r) {
      const StoreT* row = G.base + (size_t)(pv0 + r) * G.pitch + pu0;
      for (int cc = lane; cc < pw; cc += 32) patch[r * P + cc] = ld(row + cc);
    }
  }
  __syncwarp();
  auto at = [&](int u, int v) -> float { return staged ? patch[(v - pv0) * P + (u - pu0)] : G.at(u, v); };
  // central differences, clamp-to-edge
  auto grad = [&](int u, int v, float& gx, float& gy) {
    gx = at(min(u + 1, G.W - 1), v) - at(max(u - 1, 0), v);
    gy = at(u, min(v + 1, G.H - 1)) - at(u, max(v - 1, 0));
  };

  // ---- stage A
  float thetas[kMaxOri];
  int n_ori = 1;
  thetas[0] = 0.0f;
  if (!a.upright) {
    for (int b = lane; b < 36; b += 32) ho[b] = 0u;
    __syncwarp();
    const float R2 = Ro * Ro;
    const float sw = a.ori_wsig * c.so;
    const float inv2 = 1.0f / (2.0f * sw * sw);
    const int ou0 = max((int)ceilf(c.xo - Ro), 0), ou1 = min((int)floorf(c.xo + Ro), G.W - 1);
    const int ov0 = max((int)ceilf(c.yo - Ro), 0), ov1 = min((int)floorf(c.yo + Ro), G.H - 1);
    const float osc = vote_scale(max(ou1 - ou0 + 1, 0) * max(ov1 - ov0 + 1, 0));
    for_box(ou0, ov0, ou1 - ou0 + 1, ov1 - ov0 + 1, lane, [&](int u, int v) {
      const float du = (float)u - c.xo, dv = (float)v - c.yo;
      const float d2 = du * du + dv * dv;
      if (!(d2 < R2)) return;
      float gx, gy;
      grad(u, v, gx, gy);
      const float w = sqrtf(gx * gx + gy * gy) * expf(-d2 * inv2);
      const float f = atan2f(gy, gx) * (36.0f / kTwoPi);
      int b = (int)floorf(f);
      b = ((b % 36) + 36) % 36;
      vote(ho + b, w, osc);
    });
    __syncwarp();
    // every lane reads the 36 sums; the peak search is uniform over the warp
    float h[36];
#pragma unroll
    for (int b = 0; b < 36; ++b) h[b] = (float)ho[b] / osc;
    float mx = 0.0f;
#pragma unroll
    for (int b = 0; b < 36; ++b) mx = fmaxf(mx, h[b]);
    float pv[kMaxOri];
    n_ori = 0;
#pragma unroll
    for (int b = 0; b < 36; ++b) {
      const float l = h[(b + 35) % 36], cc = h[b], r = h[(b + 1) % 36];
      if (!(cc > l && cc > r)) continue;
      if (!(cc > a.ori_ratio * mx)) continue;
      const float off = 0.5f * (l - r) / (l - 2.0f * cc + r);
      float t = kTwoPi * ((float)b + 0.5f + off) / 36.0f;
      if (t >= kTwoPi) t -= kTwoPi;
      if (t < 0.0f) t += kTwoPi;
      // keep the max_ori largest, by (value desc, bin asc)
      int j = n_ori < a.max_ori ? n_ori++ : a.max_ori;
      while (j > 0 && cc > pv[j - 1]) {
        if (j < a.max_ori) {
          pv[j] = pv[j - 1];
          thetas[j] = thetas[j - 1];
        }
        --j;
      }
      if (j < a.max_ori) {
        pv[j] = cc;
        thetas[j] = t;
      }
    }
  }
  if (lane == 0) a.ori_count[slot] = n_ori;

  // ---- stage B, per orientation
  const float Rd2 = Rd * Rd;
  const float inv_cs = 1.0f / (a.cell_side * c.so);
  const float inv2w = 1.0f / (2.0f * a.desc_wsig * a.desc_wsig);
  const int du0 = max((int)ceilf(c.xo - Rd), 0), du1 = min((int)floorf(c.xo + Rd), G.W - 1);
  const int dv0 = max((int)ceilf(c.yo - Rd), 0), dv1 = min((int)floorf(c.yo + Rd), G.H - 1);
  const float dsc = vote_scale(max(du1 - du0 + 1, 0) * max(dv1 - dv0 + 1, 0));
  const size_t out0 = (size_t)slot * a.max_ori;
  for (int j = 0; j < n_ori; ++j) {
    const float theta = thetas[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) hd[lane + 32 * q] = 0u;
    __syncwarp();
    float st, ct;
    sincosf(theta, &st, &ct);
    for_box(du0, dv0, du1 - du0 + 1, dv1 - dv0 + 1, lane, [&](int u, int v) {
      const float du = (float)u - c.xo, dv = (float)v - c.yo;
      if (!(du * du + dv * dv < Rd2)) return;
      const float xr = (ct * du + st * dv) * inv_cs;
      const float yr = (-st * du + ct * dv) * inv_cs;
      float gx, gy;
      grad(u, v, gx, gy);
      const float mag = sqrtf(gx * gx + gy * gy);
      float ang = atan2f(gy, gx) - theta;
      while (ang < 0.0f) ang += kTwoPi;
      while (ang >= kTwoPi) ang -= kTwoPi;
      float ob = ang * (8.0f / kTwoPi);
      if (ob >= 8.0f) ob -= 8.0f;
      const float w = mag * expf(-(xr * xr + yr * yr) * inv2w);
      const float cx = xr + 1.5f, cy = yr + 1.5f;
      const float fx0 = floorf(cx), fy0 = floorf(cy), fo0 = floorf(ob);
      const float fx = cx - fx0, fy = cy - fy0, fo = ob - fo0;
      const int x0 = (int)fx0, y0 = (int)fy0, o0 = (int)fo0;
#pragma unroll
      for (int iy = 0; iy < 2; ++iy) {
        const int yy = y0 + iy;
        if (yy < 0 || yy > 3) continue;
        const float wy = w * (iy ? fy : 1.0f - fy);
#pragma unroll
        for (int ix = 0; ix < 2; ++ix) {
          const int xx = x0 + ix;
          if (xx < 0 || xx > 3) continue;
          const float wxy = wy * (ix ? fx : 1.0f - fx);
          const int cb = (yy * 4 + xx) * 8;
          vote(hd + cb + (o0 & 7), wxy * (1.0f - fo), dsc);
          vote(hd + cb + ((o0 + 1) & 7), wxy * fo, dsc);
        }
      }
    });
    __syncwarp();
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (float)hd[lane + 32 * q] / dsc;
    float n2 = warp_sum(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
    if (n2 > 0.0f) {
      const float inv = 1.0f / sqrtf(n2);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = fminf(v[q] * inv, 0.2f);
      n2 = warp_sum(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
      const float inv2 = 1.0f / sqrtf(n2);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] *= inv2;
    }
    float* d = a.stage_desc + (out0 + j) * 128;
#pragma unroll
    for (int q = 0; q < 4; ++q) d[lane + 32 * q] = v[q];
    if (lane == 0) {
      const float s = (float)(1 << c.octave);
      cdvs_keypoint kp;
      kp.x = c.xo * s;
      kp.y = c.yo * s;
      kp.sigma = c.so * s;
      kp.theta = theta;
      kp.response = c.resp;
      kp.p_ss = c.pss;
      kp.ratio = c.ratio;
      kp.octave = c.octave;
      kp.scale_idx = (int16_t)k;
      kp.type = c.type;
      kp.reserved = 0;
      kp.image = img;
      kp.parent_id = rank;
      a.stage_kp[out0 + j] = kp;
    }
    __syncwarp();
  }
}

// ---- packing: record offsets of every (image, rank, copy) in batch order
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const __grid_constant__ DescribeArgs a,
                                                            int* slot_off) {
  __shared__ int warp_sums[33];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = a.n_images * a.N;
  const int per = (S + kScanThreads - 1) / kScanThreads;
  const int b0 = min(tid * per, S), b1 = min(b0 + per, S);
  auto count_of = [&](int slot) {
    const int img = slot / a.N, rank = slot - img * a.N;
    return rank < a.sel_count[img] ? a.ori_count[slot] : 0;
  };
  int local = 0;
  for (int s = b0; s < b1; ++s) local += count_of(s);
  int incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = warp_sums[lane];
    int wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += v;
    }
    warp_sums[lane] = wi - w;
    if (lane == 31) warp_sums[32] = wi;
  }
  __syncthreads();
  int run = warp_sums[warp] + incl - local;
  const int total = warp_sums[32];
  const int cap = a.kp_capacity;
  for (int s = b0; s < b1; ++s) {
    const int c = count_of(s);
    slot_off[s] = run;
    for (int j = 0; j < c; ++j)
      if (run + j < cap) a.rec_map[run + j] = s * kMaxOri + j;
    run += c;
  }
  if (tid == 0) slot_off[S] = total;
  __syncthreads();
  for (int i = tid; i < a.n_images; i += kScanThreads) {
    const int beg = min(slot_off[i * a.N], cap), end = min(slot_off[(i + 1) * a.N], cap);
    a.kp_count[i] = end - beg;
  }
  if (tid == 0) {
    *a.rec_total = min(total, cap);
    if (total > cap) atomicOr(a.status, kStatusOutTruncated);
  }
}

// ---- packed output: record r of the batch comes from staging slot rec_map[r]
__global__ void __launch_bounds__(256) copy_kernel(const __grid_constant__ DescribeArgs a) {
  const int lane = threadIdx.x & 31;
  const int total = *a.rec_total;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < total; r += (gridDim.x * blockDim.x) >> 5) {
    const int m = a.rec_map[r];
    const size_t src = (size_t)(m / kMaxOri) * a.max_ori + (m % kMaxOri);
    reinterpret_cast<float4*>(a.desc_out + (size_t)r * 128)[lane] =
        reinterpret_cast<const float4*>(a.stage_desc + src * 128)[lane];
    if (lane == 0) a.kp_out[r] = a.stage_kp[src];
  }
}

template <typename StoreT>
__global__ void levels_to_f32_kernel(const StoreT* src, int W, int H, int lpitch, float* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x < W && y < H) out[(size_t)y * W + x] = ld(src + (size_t)y * lpitch + x);
}

}  // namespace

size_t describe_smem_bytes(int patch_side) {
  return (size_t)kFWarps * ((size_t)patch_side * patch_side * sizeof(float) + (36 + 128) * sizeof(unsigned));
}

cudaError_t launch_describe(const DescribeArgs& a, int storage, cudaStream_t s) {
  const int slots = a.n_images * a.N;
  if (slots <= 0) return cudaSuccess;
  const int grid = (slots + kFWarps - 1) / kFWarps;
  const size_t smem = describe_smem_bytes(a.patch_side);
  cudaError_t e;
  if (storage == CDVS_STORAGE_FP16) {
    e = cudaFuncSetAttribute(describe_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    describe_kernel<__half><<<grid, kFWarps * 32, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(describe_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    describe_kernel<float><<<grid, kFWarps * 32, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// The slot offsets live right after the record map's kp_capacity entries
// (the caller allocates kp_capacity + n_images * N + 1 ints).
cudaError_t launch_pack(const DescribeArgs& a, cudaStream_t s) {
  if (a.n_images * a.N <= 0) return cudaSuccess;
  scan_kernel<<<1, kScanThreads, 0, s>>>(a, a.rec_map + a.kp_capacity);
  return cudaGetLastError();
}

cudaError_t launch_copy(const DescribeArgs& a, int n_sms, cudaStream_t s) {
  if (a.n_images * a.N <= 0) return cudaSuccess;
  copy_kernel<<<n_sms * 8, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_levels_to_f32(const ImgPlan* plans, int img, const void* levels, int storage,
                                 int octave, int k, int W, int H, long long off, int lpitch,
                                 float* out, cudaStream_t s) {
  (void)plans;
  (void)img;
  (void)octave;
  (void)k;
  dim3 grid((W + 255) / 256, H);
  if (storage == CDVS_STORAGE_FP16)
    levels_to_f32_kernel<__half><<<grid, 256, 0, s>>>(reinterpret_cast<const __half*>(levels) + off, W, H,
                                                      lpitch, out);
  else
    levels_to_f32_kernel<float><<<grid, 256, 0, s>>>(reinterpret_cast<const float*>(levels) + off, W, H,
                                                     lpitch, out);
  return cudaGetLastError();
}

}  // namespace cdvs
