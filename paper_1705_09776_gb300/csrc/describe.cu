// describe.cu -- Alg. 2 on the GPU: dominant orientations (stage A) and
// 128-D descriptors (stage B), then the packing of the (point, orientation)
// records of the whole batch.
//
// One warp per selected point, persistent warps: the warp stages the point's
// patch of its Gaussian level in shared memory (4-byte asynchronous copies,
// all in flight at once, the image border replicated), builds the 36-bin
// orientation histogram from it, finds the orientations, and for each one
// builds the 4x4x8 descriptor histogram.  Each lane walks a contiguous run of
// the sampling disc's pixels (rows clipped to the disc, so no lane idles on
// the box corners, and the 32 runs are spread over the disc, so concurrent
// votes rarely hit the same bin).  Votes go to a per-warp histogram with
// 32-bit integer atomics on a power-of-two fixed-point scale: integer addition
// is associative, so the sums do not depend on the order in which lanes land.
#include <algorithm>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {


__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }

// A level in the image's frame: W x H, pixel (x, y) at base[y * sy + x * sx]
// -- (sx, sy) = (1, pitch), or (pitch, 1) for an octave stored transposed.
template <typename StoreT>
struct LevelView {
  const StoreT* base;
  int W, H, sx, sy;
  __device__ __forceinline__ float at(int x, int y) const { return ld(base + (size_t)y * sy + (size_t)x * sx); }
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
  v.W = op.tr ? op.H : op.W;
  v.H = op.tr ? op.W : op.H;
  v.sx = op.tr ? op.lpitch : 1;
  v.sy = op.tr ? 1 : op.lpitch;
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
// weights <= 1 with |g| <= 255 * sqrt(2) < 512, and a bin takes at most one
// vote per pixel, so n pixels keep a bin below 512 n; the scale is the
// largest power of two <= 2^13 that keeps 512 (n + 1) below 2^32.  The scaled
// vote is rounded by adding 1.5 * 2^23 in FP32 (exact for values below 2^22)
// and reading the mantissa.
constexpr int kFWarps = 8;
// Descriptor bins: cell (y0, x0) and orientation o at y0 * kCellRow + x0 * 8 + o.
// A cell row takes 36 words, not 32.  Lane l's run of disc pixels starts about
// one disc row below lane l-1's, so at any step a warp's lanes lie on a line
// across the disc, in several cell rows; with 32-word rows the same cell
// column and orientation of every cell row would share a bank.
constexpr int kCellRow = 36;
constexpr int kHdWords = 4 * kCellRow;
__device__ __forceinline__ int hd_index(int b) { return b + (b >> 5) * (kCellRow - 32); }
constexpr float kPi = 3.14159265358979f;
constexpr float kHalfPi = 1.57079632679490f;
constexpr float kLog2e = 1.44269504088896f;

__device__ __forceinline__ float vote_scale(int n_pixels) {
  int sh = 13;
  while (sh > 0 && (512.0 * (double)(n_pixels + 1)) * (double)(1 << sh) >= 4294967296.0) --sh;
  return (float)(1 << sh);
}

__device__ __forceinline__ void vote(unsigned* h, float w, float scale) {
  const unsigned q = (unsigned)(__float_as_int(fmaf(w, scale, 12582912.0f)) - 0x4B400000);
  atomicAdd(h, q);
}

// The approximate hardware instructions (PTX ex2.approx, sqrt.approx,
// rcp.approx; relative errors of a few FP32 ulps): the weights they feed are
// smooth in their inputs, so these errors stay far below the parity tolerance.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// atan2(y, x) in [-pi, pi]: t = min(|x|, |y|) / max(|x|, |y|) in [0, 1],
// atan(t) = t P(t^2) with the degree-15 near-minimax odd polynomial printed by
// fit_atan.py (|error| < 1.2e-7 rad in FP32), then the octant: pi/2 - r when
// |y| > |x|, pi - r when x < 0, and the sign of y.  Gradients below 1e-30 in
// both components give 0 or pi; their votes weigh nothing.
__device__ __forceinline__ float atan2_poly(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float t = mx >= 1e-30f ? mn * rcp_approx(mx) : 0.0f;
  const float z = t * t;
  float p = -4.054549150e-03f;
  p = fmaf(p, z, 2.186289616e-02f);
  p = fmaf(p, z, -5.591224134e-02f);
  p = fmaf(p, z, 9.642191231e-02f);
  p = fmaf(p, z, -1.390862763e-01f);
  p = fmaf(p, z, 1.994656473e-01f);
  p = fmaf(p, z, -3.332985938e-01f);
  p = fmaf(p, z, 9.999993443e-01f);
  float r = p * t;
  r = ay > ax ? kHalfPi - r : r;
  r = x < 0.0f ? kPi - r : r;
  return copysignf(r, y);
}

// ---- sampling discs
// The pixels (u, v) with (u - xo)^2 + (v - yo)^2 < R^2, clipped to the box
// [bx0, bx1] x [by0, by1], are walked in bands of at most P rows (P = the
// warp's row-table length; one band whenever the patch is staged).  For a
// band, the warp's shared row tables hold per row r (v = v0 + r) the first
// column ru[r], the count rn[r] and the exclusive prefix rp[r] of the counts.
// The row spans come from h = sqrt(R^2 - dv^2) (pixels strictly inside); a
// pixel within FP32 rounding of the circle may fall on either side.
struct Disc {
  int v0, nr, total;
};

__device__ __forceinline__ void disc_rows(float yo, float R, int by0, int by1, int& v0, int& n) {
  v0 = max((int)ceilf(yo - R), by0);
  n = max(min((int)floorf(yo + R), by1) - v0 + 1, 0);
}

__device__ __forceinline__ Disc build_band(float xo, float yo, float R2, int bx0, int bx1, int v0, int nr,
                                           int* ru, int* rn, int* rp, int lane) {
  Disc d;
  d.v0 = v0;
  d.nr = nr;
  int carry = 0;
  for (int r0 = 0; r0 < nr; r0 += 32) {
    const int r = r0 + lane;
    int n = 0;
    if (r < nr) {
      const float dv = (float)(v0 + r) - yo;
      const float h2 = R2 - dv * dv;
      int lo = 0;
      if (h2 > 0.0f) {
        const float h = sqrtf(h2);
        lo = max((int)floorf(xo - h) + 1, bx0);
        const int hi = min((int)ceilf(xo + h) - 1, bx1);
        n = max(hi - lo + 1, 0);
      }
      ru[r] = lo;
      rn[r] = n;
    }
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (r < nr) rp[r] = carry + incl - n;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  d.total = carry;
  __syncwarp();
  return d;
}

// Lane l visits the disc pixels [l T / 32, (l + 1) T / 32) in row order and
// calls f(u, v) for each.
template <typename F>
__device__ __forceinline__ void for_disc(const Disc& d, const int* ru, const int* rn, const int* rp, int lane,
                                         F&& f) {
  const int i0 = (d.total * lane) >> 5, i1 = (d.total * (lane + 1)) >> 5;
  if (i0 >= i1) return;
  // the row holding pixel i0: the last row r with rp[r] <= i0 (an empty row
  // shares its prefix with the next one, which then wins)
  int lo = 0, hi = d.nr;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (rp[mid] <= i0) lo = mid;
    else hi = mid;
  }
  int r = lo;
  int u = ru[r] + (i0 - rp[r]);
  int rem = rn[r] - (i0 - rp[r]);
  for (int i = i0; i < i1; ++i) {
    f(u, d.v0 + r);
    ++u;
    if (--rem == 0 && i + 1 < i1) {
      // pixels remain, so a non-empty row follows within the table
      do {
        ++r;
      } while (r + 1 < d.nr && rn[r] == 0);
      u = ru[r];
      rem = rn[r];
    }
  }
}

// Every pixel of the disc of radius R, band by band: f(u, v) on each.
template <typename F>
__device__ __forceinline__ void for_each_disc_pixel(float xo, float yo, float R, int bx0, int bx1, int by0,
                                                    int by1, int P, int* ru, int* rn, int* rp, int lane, F&& f) {
  int v0, n;
  disc_rows(yo, R, by0, by1, v0, n);
  for (int b0 = 0; b0 < n; b0 += P) {
    const Disc d = build_band(xo, yo, R * R, bx0, bx1, v0 + b0, min(P, n - b0), ru, rn, rp, lane);
    for_disc(d, ru, rn, rp, lane, f);
    __syncwarp();  // the row tables are rebuilt for the next band
  }
}

// Central-difference gradients, clamp-to-edge.  PatchSrc reads the staged
// patch, whose one-pixel ring around the sampling box already holds the
// replicated edge, so it needs no clamps; LevelSrc reads the level itself.
struct PatchSrc {
  const float* p;  // patch element (pu0, pv0)
  int P, pu0, pv0;
  __device__ __forceinline__ void grad(int u, int v, float& gx, float& gy) const {
    const float* q = p + (v - pv0) * P + (u - pu0);
    gx = q[1] - q[-1];
    gy = q[P] - q[-P];
  }
};

template <typename StoreT>
struct LevelSrc {
  LevelView<StoreT> G;
  __device__ __forceinline__ void grad(int u, int v, float& gx, float& gy) const { G.grad(u, v, gx, gy); }
};

// ---- Alg. 2 for one point.  Stage A: 36-bin histogram of atan2(gy, gx)
// over the disc of radius ori_radius * sigma, weight
// |g| exp(-d^2 / (2 (ori_wsig sigma)^2)); orientations at bins strictly above
// both circular neighbours and above ori_ratio * max, refined by a parabola
// through three bins, in order of bin value.  Stage B, per orientation: 4x4
// cells of side cell_side * sigma in the frame rotated by -theta, 8 bins of
// the gradient angle relative to theta, trilinear votes weighted by
// |g| exp(-(u^2+v^2) / (2 desc_wsig^2)) ((u, v) in cells; the rotation keeps
// u^2 + v^2 = d^2 / cell^2) over the disc of radius desc_radius * sigma;
// L2-normalise, clamp at 0.2, renormalise.  Records and descriptors go to the
// point's staging slots (max_ori each).
template <typename Src>
__device__ __forceinline__ void describe_point(const DescribeArgs& a, const Cand& c, int slot, int img, int rank,
                                               int k, const Src& src, int bx0, int bx1, int by0, int by1, int P,
                                               unsigned* ho, unsigned* hd, float* thetas, int* ru, int* rn, int* rp,
                                               int lane) {
  // vote scales from the box area, which bounds the pixel count of any disc
  const float osc = vote_scale((bx1 - bx0 + 1) * (by1 - by0 + 1)), dsc = osc;
  int n_ori = 1;
  if (lane == 0) thetas[0] = 0.0f;
  if (!a.upright) {
    for (int b = lane; b < 36; b += 32) ho[b] = 0u;
    __syncwarp();
    const float sw = a.ori_wsig * c.so;
    const float kA = -kLog2e / (2.0f * sw * sw);
    for_each_disc_pixel(c.xo, c.yo, a.ori_radius * c.so, bx0, bx1, by0, by1, P, ru, rn, rp, lane,
                        [&](int u, int v) {
      const float du = (float)u - c.xo, dv = (float)v - c.yo;
      float gx, gy;
      src.grad(u, v, gx, gy);
      const float w = sqrt_approx(gx * gx + gy * gy) * ex2_approx((du * du + dv * dv) * kA);
      int b = (int)floorf(atan2_poly(gy, gx) * (36.0f / (2.0f * kPi)));
      b += b < 0 ? 36 : 0;
      b -= b >= 36 ? 36 : 0;
      vote(ho + b, w, osc);
    });
    __syncwarp();
    // peaks: lane b (and b + 32) takes bin b; a peak's place among the
    // orientations is its rank by (value desc, bin asc)
    const float inv_osc = 1.0f / osc;
    float hv[2], mx = 0.0f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int b = lane + 32 * q;
      hv[q] = b < 36 ? (float)ho[b] * inv_osc : 0.0f;
      mx = fmaxf(mx, hv[q]);
    }
    mx = warp_max(mx);
    bool pk[2];
    float th[2];
    unsigned peaks[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int b = lane + 32 * q;
      pk[q] = false;
      th[q] = 0.0f;
      if (b < 36) {
        const float l = (float)ho[b == 0 ? 35 : b - 1] * inv_osc, cc = hv[q];
        const float r = (float)ho[b == 35 ? 0 : b + 1] * inv_osc;
        pk[q] = cc > l && cc > r && cc > a.ori_ratio * mx;
        const float off = 0.5f * (l - r) / (l - 2.0f * cc + r);
        float t = 2.0f * kPi * ((float)b + 0.5f + off) / 36.0f;
        if (t >= 2.0f * kPi) t -= 2.0f * kPi;
        if (t < 0.0f) t += 2.0f * kPi;
        th[q] = t;
      }
      peaks[q] = __ballot_sync(0xffffffffu, pk[q]);
    }
    n_ori = min(__popc(peaks[0]) + __popc(peaks[1]), a.max_ori);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!pk[q]) continue;
      const int b = lane + 32 * q;
      int rank = 0;
      for (int m = 0; m < 2; ++m)
        for (unsigned bits = peaks[m]; bits; bits &= bits - 1) {
          const int b2 = __ffs(bits) - 1 + 32 * m;
          const float v2 = (float)ho[b2] * inv_osc;
          rank += v2 > hv[q] || (v2 == hv[q] && b2 < b);
        }
      if (rank < a.max_ori) thetas[rank] = th[q];
    }
    __syncwarp();
  }
  if (lane == 0) a.ori_count[slot] = n_ori;

  // ---- stage B, per orientation
  const float inv_cs = 1.0f / (a.cell_side * c.so);
  const float kB = -kLog2e * inv_cs * inv_cs / (2.0f * a.desc_wsig * a.desc_wsig);
  const size_t out0 = (size_t)slot * a.max_ori;
  __syncwarp();
  for (int j = 0; j < n_ori; ++j) {
    const float theta = thetas[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) hd[hd_index(lane + 32 * q)] = 0u;
    __syncwarp();
    float st, ct;
    sincosf(theta, &st, &ct);
    const float cc_ = ct * inv_cs, sc_ = st * inv_cs;
    for_each_disc_pixel(c.xo, c.yo, a.desc_radius * c.so, bx0, bx1, by0, by1, P, ru, rn, rp, lane,
                        [&](int u, int v) {
      const float du = (float)u - c.xo, dv = (float)v - c.yo;
      const float xr = fmaf(cc_, du, sc_ * dv);
      const float yr = fmaf(cc_, dv, -sc_ * du);
      float gx, gy;
      src.grad(u, v, gx, gy);
      const float w = sqrt_approx(gx * gx + gy * gy) * ex2_approx((du * du + dv * dv) * kB);
      float ob = (atan2_poly(gy, gx) - theta) * (8.0f / (2.0f * kPi));
      ob += ob < 0.0f ? 8.0f : 0.0f;
      ob += ob < 0.0f ? 8.0f : 0.0f;
      ob -= ob >= 8.0f ? 8.0f : 0.0f;
      const float cx = xr + 1.5f, cy = yr + 1.5f;
      const float fx0 = floorf(cx), fy0 = floorf(cy), fo0 = floorf(ob);
      const float fx = cx - fx0, fy = cy - fy0, fo = ob - fo0;
      const int x0 = (int)fx0, y0 = (int)fy0, o0 = (int)fo0;
      // the scaled orientation shares, then one multiply-add per vote (the
      // vote wxy * a, a already scaled); the 2 x 2 cells as straight-line
      // code, each vote pair guarded by its cell lying in the 4 x 4 grid
      // (x0 and y0 are in -1 .. 3)
      const float ws = w * dsc;
      const float a0 = ws * (1.0f - fo), a1 = ws * fo;
      const bool x0ok = x0 >= 0, x1ok = x0 <= 2, y0ok = y0 >= 0, y1ok = y0 <= 2;
      const float wy0 = 1.0f - fy, wx0 = 1.0f - fx;
      const int cb = y0 * kCellRow + x0 * 8;
      const int i0 = (o0 & 7) + cb, i1 = ((o0 + 1) & 7) + cb;
      if (y0ok && x0ok) {
        vote(hd + i0, wy0 * wx0, a0);
        vote(hd + i1, wy0 * wx0, a1);
      }
      if (y0ok && x1ok) {
        vote(hd + i0 + 8, wy0 * fx, a0);
        vote(hd + i1 + 8, wy0 * fx, a1);
      }
      if (y1ok && x0ok) {
        vote(hd + i0 + kCellRow, fy * wx0, a0);
        vote(hd + i1 + kCellRow, fy * wx0, a1);
      }
      if (y1ok && x1ok) {
        vote(hd + i0 + kCellRow + 8, fy * fx, a0);
        vote(hd + i1 + kCellRow + 8, fy * fx, a1);
      }
    });
    __syncwarp();
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (float)hd[hd_index(lane + 32 * q)] / dsc;
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
    float* dd = a.stage_desc + (out0 + j) * 128;
#pragma unroll
    for (int q = 0; q < 4; ++q) dd[lane + 32 * q] = v[q];
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

// Points whose box does not fit the patch read the level directly; kept out
// of line so the kernel's hot code stays small.
template <typename StoreT>
__device__ __noinline__ void describe_point_unstaged(const DescribeArgs& a, const Cand& c, int slot, int img,
                                                     int rank, int k, const LevelView<StoreT>& G, int bx0, int bx1,
                                                     int by0, int by1, int P, unsigned* ho, unsigned* hd,
                                                     float* thetas, int* ru, int* rn, int* rp, int lane) {
  LevelSrc<StoreT> src{G};
  describe_point(a, c, slot, img, rank, k, src, bx0, bx1, by0, by1, P, ho, hd, thetas, ru, rn, rp, lane);
}

// 4 bytes global -> shared without passing through registers
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}

// Patch rows pv0 .. pv0 + ph - 1, columns pu0 .. pu0 + pw - 1 of the level
// (image frame), clamped to the image, into patch[r * P + c].  The lanes walk
// along the stored rows: image rows, or image columns of a transposed octave.
__device__ __forceinline__ void stage_patch(const LevelView<float>& G, int pu0, int pv0, int pw, int ph, int P,
                                            float* patch, int lane) {
  if (G.sx == 1) {
    for (int r = 0; r < ph; ++r) {
      const float* row = G.base + (size_t)min(max(pv0 + r, 0), G.H - 1) * G.sy;
      for (int cc = lane; cc < pw; cc += 32) cp_async4(patch + r * P + cc, row + min(max(pu0 + cc, 0), G.W - 1));
    }
  } else {
    for (int cc = 0; cc < pw; ++cc) {
      const float* col = G.base + (size_t)min(max(pu0 + cc, 0), G.W - 1) * G.sx;
      for (int r = lane; r < ph; r += 32) cp_async4(patch + r * P + cc, col + min(max(pv0 + r, 0), G.H - 1));
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}
__device__ __forceinline__ void stage_patch(const LevelView<__half>& G, int pu0, int pv0, int pw, int ph, int P,
                                            float* patch, int lane) {
  if (G.sx == 1) {
    for (int r = 0; r < ph; ++r) {
      const __half* row = G.base + (size_t)min(max(pv0 + r, 0), G.H - 1) * G.sy;
      for (int cc = lane; cc < pw; cc += 32) patch[r * P + cc] = ld(row + min(max(pu0 + cc, 0), G.W - 1));
    }
  } else {
    for (int cc = 0; cc < pw; ++cc) {
      const __half* col = G.base + (size_t)min(max(pu0 + cc, 0), G.W - 1) * G.sx;
      for (int r = lane; r < ph; r += 32) patch[r * P + cc] = ld(col + min(max(pv0 + r, 0), G.H - 1));
    }
  }
}

// Persistent warps claim the group's slots one at a time from its counter
// (zeroed before every call), so a warp that drew small points takes more of
// them and the grid finishes together.
template <typename StoreT>
__global__ void __launch_bounds__(kFWarps * 32, 3) describe_kernel(const __grid_constant__ DescribeArgs a) {
  extern __shared__ float4 smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = a.patch_side;
  float* patch = reinterpret_cast<float*>(smem4) + (size_t)warp * P * P;
  unsigned* hist = reinterpret_cast<unsigned*>(reinterpret_cast<float*>(smem4) + (size_t)kFWarps * P * P) +
                   warp * (36 + kHdWords + kMaxOri + 3 * P);
  unsigned* ho = hist;        // 36 orientation bins
  unsigned* hd = hist + 36;   // 128 descriptor bins (at hd_index)
  float* thetas = reinterpret_cast<float*>(hist + 36 + kHdWords);  // the point's orientations
  int* ru = reinterpret_cast<int*>(hist + 36 + kHdWords + kMaxOri);  // disc row tables, P rows each
  int* rn = ru + P;
  int* rp = rn + P;
  const int S0 = a.img_begin * a.N, S1 = a.img_end * a.N;
  for (;;) {
    int slot = 0;
    if (lane == 0) slot = S0 + (int)atomicAdd(a.claim, 1u);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= S1) break;
    const int img = slot / a.N, rank = slot - img * a.N;
    if (rank >= a.sel_count[img]) continue;
    const Cand c = a.sel[slot];
    const int k = desc_level(c.so, a.sigma0);
    const LevelView<StoreT> G = level_of<StoreT>(a, img, c.octave, k);
    // the sampling box of both discs, clipped to the image
    const float R = fmaxf(a.desc_radius * c.so, a.upright ? 0.0f : a.ori_radius * c.so);
    const int bx0 = max((int)ceilf(c.xo - R), 0), bx1 = min((int)floorf(c.xo + R), G.W - 1);
    const int by0 = max((int)ceilf(c.yo - R), 0), by1 = min((int)floorf(c.yo + R), G.H - 1);
    // the patch: the box and a one-pixel ring (edge replicated)
    const int pu0 = bx0 - 1, pv0 = by0 - 1;
    const int pw = bx1 - bx0 + 3, ph = by1 - by0 + 3;
    if (pw <= P && ph <= P) {
      stage_patch(G, pu0, pv0, pw, ph, P, patch, lane);
      __syncwarp();
      PatchSrc src{patch, P, pu0, pv0};
      describe_point(a, c, slot, img, rank, k, src, bx0, bx1, by0, by1, P, ho, hd, thetas, ru, rn, rp, lane);
    } else {
      describe_point_unstaged<StoreT>(a, c, slot, img, rank, k, G, bx0, bx1, by0, by1, P, ho, hd, thetas, ru, rn,
                                      rp, lane);
    }
    __syncwarp();  // the patch and tables are rewritten for the next point
  }
}

// ---- packing.  Records go out in batch order: image, then rank, then copy.
// scan_kernel, per image group: one warp per image writes, per slot, the
// offset of its first record within the image (local_off) and the image's
// record count (img_tot); the CTA that finishes last (the group's counter,
// zeroed before every call) scans the group's image counts from the group's
// first record (base_in) into img_off and the per-image counts clipped to the
// capacity, and writes the next group's first record (base_out); the last
// group also writes the batch total.
constexpr int kPackWarps = 8;

__global__ void __launch_bounds__(kPackWarps * 32) scan_kernel(const __grid_constant__ DescribeArgs a,
                                                               int* local_off, int* img_tot, int* img_off) {
  __shared__ int is_last;
  __shared__ int warp_sums[kPackWarps * 32 / 32 + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int img = a.img_begin + blockIdx.x * kPackWarps + warp;
  if (img < a.img_end) {
    const int cnt = a.sel_count[img];
    const int per = (a.N + 31) / 32;
    const int r0 = min(lane * per, a.N), r1 = min(r0 + per, a.N);
    const int* oc = a.ori_count + (size_t)img * a.N;
    int local = 0;
    for (int r = r0; r < r1; ++r) local += r < cnt ? oc[r] : 0;
    int incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    int run = incl - local;
    int* lo = local_off + (size_t)img * a.N;
    for (int r = r0; r < r1; ++r) {
      lo[r] = run;
      run += r < cnt ? oc[r] : 0;
    }
    if (lane == 31) img_tot[img] = incl;
  }
  // the last CTA to arrive sees every image count
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(a.scan_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const int n = a.img_end - a.img_begin;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int i0 = a.img_begin + min((int)threadIdx.x * per, n), i1 = min(i0 + per, a.img_end);
  int local = 0;
  for (int i = i0; i < i1; ++i) local += __ldcg(img_tot + i);
  int incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kPackWarps; ++w) {
      const int v = warp_sums[w];
      warp_sums[w] = t;
      t += v;
    }
    warp_sums[kPackWarps] = t;
  }
  __syncthreads();
  const int cap = a.kp_capacity;
  const int base = __ldcg(a.base_in);
  int run = base + warp_sums[warp] + incl - local;
  for (int i = i0; i < i1; ++i) {
    const int c = __ldcg(img_tot + i);
    img_off[i] = run;
    a.kp_count[i] = min(run + c, cap) - min(run, cap);
    run += c;
  }
  if (threadIdx.x == 0) {
    const int total = base + warp_sums[kPackWarps];
    img_off[a.img_end] = total;
    *a.base_out = total;
    if (a.last_group) {
      *a.rec_total = min(total, cap);
      if (total > cap) atomicOr(a.status, kStatusOutTruncated);
    }
  }
}

// ---- packed output: one warp per slot copies its records from the staging
// slots to their batch positions (records past the capacity are dropped)
__global__ void __launch_bounds__(256) copy_kernel(const __grid_constant__ DescribeArgs a, const int* local_off,
                                                   const int* img_off) {
  const int lane = threadIdx.x & 31;
  const int S0 = a.img_begin * a.N, S1 = a.img_end * a.N;
  const int cap = a.kp_capacity;
  for (int s = S0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); s < S1; s += (gridDim.x * blockDim.x) >> 5) {
    const int img = s / a.N, rank = s - img * a.N;
    if (rank >= a.sel_count[img]) continue;
    const int n = a.ori_count[s];
    const int base = img_off[img] + local_off[s];
    for (int j = 0; j < n && base + j < cap; ++j) {
      const size_t src = (size_t)s * a.max_ori + j, dst = (size_t)(base + j);
      reinterpret_cast<float4*>(a.desc_out + dst * 128)[lane] =
          reinterpret_cast<const float4*>(a.stage_desc + src * 128)[lane];
      if (lane == 0) a.kp_out[dst] = a.stage_kp[src];
    }
  }
}

template <typename StoreT>
__global__ void levels_to_f32_kernel(const StoreT* src, int Wi, int Hi, int tr, int lpitch, float* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;  // image frame
  const int y = blockIdx.y;
  if (x < Wi && y < Hi) out[(size_t)y * Wi + x] = ld(tr ? src + (size_t)x * lpitch + y : src + (size_t)y * lpitch + x);
}

}  // namespace

size_t describe_smem_bytes(int patch_side) {
  return (size_t)kFWarps * ((size_t)patch_side * patch_side * sizeof(float) +
                            (36 + kHdWords + kMaxOri + 3 * (size_t)patch_side) * sizeof(unsigned));
}

// Persistent grid: as many CTAs as fit on the SMs at once (never more than
// there are slots for).
cudaError_t launch_describe(const DescribeArgs& a, int storage, int n_sms, cudaStream_t s) {
  const int slots = (a.img_end - a.img_begin) * a.N;
  if (slots <= 0) return cudaSuccess;
  const size_t smem = describe_smem_bytes(a.patch_side);
  static LaunchCache cache32, cache16;
  auto go = [&](auto kernel, LaunchCache& cache) -> cudaError_t {
    int per_sm = 0;
    cudaError_t e = prepare_launch(kernel, cache, (int)smem, kFWarps * 32, &per_sm);
    if (e != cudaSuccess) return e;
    const int need = (slots + kFWarps - 1) / kFWarps;
    const int grid = std::max(1, std::min(need, std::max(per_sm, 1) * n_sms));
    kernel<<<grid, kFWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
  };
  return storage == CDVS_STORAGE_FP16 ? go(describe_kernel<__half>, cache16) : go(describe_kernel<float>, cache32);
}

// The packing scratch (rec_off) holds local_off (n_images * N ints), then
// img_tot (n_images), then img_off (n_images + 1).
cudaError_t launch_pack(const DescribeArgs& a, cudaStream_t s) {
  if (a.img_end <= a.img_begin || a.N <= 0) return cudaSuccess;
  int* local_off = a.rec_off;
  int* img_tot = local_off + (size_t)a.n_images * a.N;
  int* img_off = img_tot + a.n_images;
  scan_kernel<<<(a.img_end - a.img_begin + kPackWarps - 1) / kPackWarps, kPackWarps * 32, 0, s>>>(a, local_off, img_tot,
                                                                                     img_off);
  return cudaGetLastError();
}

cudaError_t launch_copy(const DescribeArgs& a, int n_sms, cudaStream_t s) {
  if (a.img_end <= a.img_begin || a.N <= 0) return cudaSuccess;
  const int* local_off = a.rec_off;
  const int* img_off = local_off + (size_t)a.n_images * a.N + a.n_images;
  const int slots = (a.img_end - a.img_begin) * a.N;
  const int grid = std::min((slots + 7) / 8, n_sms * 8);
  copy_kernel<<<grid, 256, 0, s>>>(a, local_off, img_off);
  return cudaGetLastError();
}

cudaError_t launch_levels_to_f32(const void* levels, int storage, int W, int H, int tr, long long off, int lpitch,
                                 float* out, cudaStream_t s) {
  const int Wi = tr ? H : W, Hi = tr ? W : H;
  dim3 grid((Wi + 255) / 256, Hi);
  if (storage == CDVS_STORAGE_FP16)
    levels_to_f32_kernel<__half><<<grid, 256, 0, s>>>(reinterpret_cast<const __half*>(levels) + off, Wi, Hi, tr,
                                                      lpitch, out);
  else
    levels_to_f32_kernel<float><<<grid, 256, 0, s>>>(reinterpret_cast<const float*>(levels) + off, Wi, Hi, tr,
                                                     lpitch, out);
  return cudaGetLastError();
}

}  // namespace cdvs
