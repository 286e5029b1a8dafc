// describe.cu -- Alg. 2 on the GPU: K5 dominant orientations (stage A),
// a scan that packs the (point, orientation) records of the whole batch, and
// K6 128-D descriptors (stage B).
//
// One warp per point (K5) and one warp per record (K6): the lanes stride
// over the pixels of the sampling disc and vote into lane-private histograms
// in shared memory laid out [bin][lane] (bank = lane, no conflicts, no
// atomics); the lane copies are summed in a fixed order, so the result does
// not depend on scheduling.
#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr float kTwoPi = 6.283185307179586f;
constexpr int kOriWarps = 8;
constexpr int kDescWarps = 4;
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

// ---- K5: 36-bin orientation histogram over the disc of radius
// ori_radius * sigma, weight |g| exp(-d^2 / (2 (ori_wsig sigma)^2)); peaks
// strictly above both circular neighbours and above ori_ratio * max, each
// refined by a parabola through three bins.
template <typename StoreT>
__global__ void __launch_bounds__(kOriWarps * 32) orient_kernel(const __grid_constant__ DescribeArgs a) {
  __shared__ float hist[kOriWarps][36][32];
  __shared__ float h36[kOriWarps][36];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = blockIdx.x * kOriWarps + warp;
  if (slot >= a.n_images * a.N) return;
  const int img = slot / a.N, rank = slot - img * a.N;
  if (rank >= a.sel_count[img]) return;
  const Cand c = a.sel[slot];
  float* th = a.ori_theta + (size_t)slot * kMaxOri;
  if (a.upright) {
    if (lane == 0) {
      th[0] = 0.0f;
      a.ori_count[slot] = 1;
    }
    return;
  }
  const int k = desc_level(c.so, a.sigma0);
  const LevelView<StoreT> G = level_of<StoreT>(a, img, c.octave, k);
  float(*hw)[32] = hist[warp];
  for (int b = 0; b < 36; ++b) hw[b][lane] = 0.0f;
  const float R = a.ori_radius * c.so, R2 = R * R;
  const float sw = a.ori_wsig * c.so;
  const float inv2 = 1.0f / (2.0f * sw * sw);
  const int u0 = max((int)ceilf(c.xo - R), 0), u1 = min((int)floorf(c.xo + R), G.W - 1);
  const int v0 = max((int)ceilf(c.yo - R), 0), v1 = min((int)floorf(c.yo + R), G.H - 1);
  const int bw = u1 - u0 + 1, bh = v1 - v0 + 1;
  if (bw > 0 && bh > 0) {
    for (int i = lane; i < bw * bh; i += 32) {
      const int vv = i / bw;
      const int v = v0 + vv, u = u0 + (i - vv * bw);
      const float du = (float)u - c.xo, dv = (float)v - c.yo;
      const float d2 = du * du + dv * dv;
      if (!(d2 < R2)) continue;
      float gx, gy;
      G.grad(u, v, gx, gy);
      const float w = sqrtf(gx * gx + gy * gy) * expf(-d2 * inv2);
      const float f = atan2f(gy, gx) * (36.0f / kTwoPi);
      int b = (int)floorf(f);
      b = ((b % 36) + 36) % 36;
      hw[b][lane] += w;
    }
  }
  __syncwarp();
  for (int b = lane; b < 36; b += 32) {
    float s = 0.0f;
    for (int l = 0; l < 32; ++l) s += hw[b][l];
    h36[warp][b] = s;
  }
  __syncwarp();
  const float* h = h36[warp];
  float mx = fmaxf(h[lane], lane < 4 ? h[32 + lane] : 0.0f);
  mx = warp_max(mx);
  if (lane == 0) {
    float pv[36], pt[36];
    int pb[36], np = 0;
    for (int b = 0; b < 36; ++b) {
      const float l = h[(b + 35) % 36], cc = h[b], r = h[(b + 1) % 36];
      if (!(cc > l && cc > r)) continue;
      if (!(cc > a.ori_ratio * mx)) continue;
      const float off = 0.5f * (l - r) / (l - 2.0f * cc + r);
      float t = kTwoPi * ((float)b + 0.5f + off) / 36.0f;
      if (t >= kTwoPi) t -= kTwoPi;
      if (t < 0.0f) t += kTwoPi;
      // insertion by (value desc, bin asc)
      int j = np++;
      while (j > 0 && (cc > pv[j - 1])) {
        pv[j] = pv[j - 1];
        pt[j] = pt[j - 1];
        pb[j] = pb[j - 1];
        --j;
      }
      pv[j] = cc;
      pt[j] = t;
      pb[j] = b;
    }
    const int n = min(np, a.max_ori);
    for (int j = 0; j < n; ++j) th[j] = pt[j];
    a.ori_count[slot] = n;
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

// ---- K6: 4x4 cells of side cell_side * sigma in the frame rotated by -theta,
// 8 orientation bins, trilinear votes weighted by |g| exp(-(u^2+v^2) /
// (2 desc_wsig^2)) with (u, v) in cells, over the disc of radius desc_radius *
// sigma; L2-normalise, clamp at 0.2, renormalise.
template <typename StoreT>
__global__ void __launch_bounds__(kDescWarps * 32) desc_kernel(const __grid_constant__ DescribeArgs a) {
  extern __shared__ float4 smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float(*hw)[32] = reinterpret_cast<float(*)[32]>(reinterpret_cast<float*>(smem4) + warp * 128 * 32);
  const int total = *a.rec_total;
  for (int r = blockIdx.x * kDescWarps + warp; r < total; r += gridDim.x * kDescWarps) {
    const int m = a.rec_map[r];
    const int slot = m / kMaxOri;
    const int img = slot / a.N, rank = slot - img * a.N;
    const Cand c = a.sel[slot];
    const float theta = a.ori_theta[m];
    const int k = desc_level(c.so, a.sigma0);
    const LevelView<StoreT> G = level_of<StoreT>(a, img, c.octave, k);
    for (int b = 0; b < 128; ++b) hw[b][lane] = 0.0f;
    const float R = a.desc_radius * c.so, R2 = R * R;
    const float inv_cs = 1.0f / (a.cell_side * c.so);
    float st, ct;
    sincosf(theta, &st, &ct);
    const float inv2w = 1.0f / (2.0f * a.desc_wsig * a.desc_wsig);
    const int u0 = max((int)ceilf(c.xo - R), 0), u1 = min((int)floorf(c.xo + R), G.W - 1);
    const int v0 = max((int)ceilf(c.yo - R), 0), v1 = min((int)floorf(c.yo + R), G.H - 1);
    const int bw = u1 - u0 + 1, bh = v1 - v0 + 1;
    if (bw > 0 && bh > 0) {
      for (int i = lane; i < bw * bh; i += 32) {
        const int vv = i / bw;
        const int v = v0 + vv, u = u0 + (i - vv * bw);
        const float du = (float)u - c.xo, dv = (float)v - c.yo;
        if (!(du * du + dv * dv < R2)) continue;
        const float xr = (ct * du + st * dv) * inv_cs;
        const float yr = (-st * du + ct * dv) * inv_cs;
        float gx, gy;
        G.grad(u, v, gx, gy);
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
            hw[cb + (o0 & 7)][lane] += wxy * (1.0f - fo);
            hw[cb + ((o0 + 1) & 7)][lane] += wxy * fo;
          }
        }
      }
    }
    __syncwarp();
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = lane + 32 * j;
      float s = 0.0f;
      for (int l = 0; l < 32; ++l) s += hw[b][l];
      v[j] = s;
    }
    float n2 = warp_sum(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
    if (n2 > 0.0f) {
      const float inv = 1.0f / sqrtf(n2);
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = fminf(v[j] * inv, 0.2f);
      n2 = warp_sum(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
      const float inv2 = 1.0f / sqrtf(n2);
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] *= inv2;
    }
    float* d = a.desc_out + (size_t)r * 128;
#pragma unroll
    for (int j = 0; j < 4; ++j) d[lane + 32 * j] = v[j];
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
      a.kp_out[r] = kp;
    }
    __syncwarp();
  }
}

template <typename StoreT>
__global__ void levels_to_f32_kernel(const StoreT* src, int W, int H, int lpitch, float* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x < W && y < H) out[(size_t)y * W + x] = ld(src + (size_t)y * lpitch + x);
}

}  // namespace

cudaError_t launch_orient(const DescribeArgs& a, int storage, cudaStream_t s) {
  const int slots = a.n_images * a.N;
  if (slots <= 0) return cudaSuccess;
  const int ob = (slots + kOriWarps - 1) / kOriWarps;
  if (storage == CDVS_STORAGE_FP16) orient_kernel<__half><<<ob, kOriWarps * 32, 0, s>>>(a);
  else orient_kernel<float><<<ob, kOriWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

// The slot offsets live right after the record map's kp_capacity entries
// (the caller allocates kp_capacity + n_images * N + 1 ints).
cudaError_t launch_pack(const DescribeArgs& a, cudaStream_t s) {
  if (a.n_images * a.N <= 0) return cudaSuccess;
  scan_kernel<<<1, kScanThreads, 0, s>>>(a, a.rec_map + a.kp_capacity);
  return cudaGetLastError();
}

cudaError_t launch_desc(const DescribeArgs& a, int storage, int n_sms, cudaStream_t s) {
  if (a.n_images * a.N <= 0) return cudaSuccess;
  const size_t dsmem = sizeof(float) * 128 * 32 * kDescWarps;
  const int db = n_sms * 4;
  cudaError_t e;
  if (storage == CDVS_STORAGE_FP16) {
    e = cudaFuncSetAttribute(desc_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
    if (e != cudaSuccess) return e;
    desc_kernel<__half><<<db, kDescWarps * 32, dsmem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(desc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
    if (e != cudaSuccess) return e;
    desc_kernel<float><<<db, kDescWarps * 32, dsmem, s>>>(a);
  }
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
