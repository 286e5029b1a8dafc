// detect.cu -- K1: one octave of interest point detection for a batch of
// images, fused in one CTA per 128x32 output tile:
//   Gaussian levels G_{o,k} (Eq. 1, Alg. 1 stage A: a pass along y then a
//   pass along x, every level filtered directly from the octave base),
//   scale-normalised 5-point LoG L_{o,k}, the per-pixel cubic in sigma of
//   Eq. 2-3, its extremum scale, the 8-neighbour test, the sub-pixel
//   refinement of Alg. 1 stage B, and warp-aggregated appends to the image's
//   candidate queue.  The same CTA stores its tile of every level (for
//   description) and, on the top level, the decimated base of the next octave
//   (Alg. 1: Downsampling G_{o,K-1} to G_{o+1,0}).
//
// Shared memory per CTA (FP32):
//   tmp  [36][128 + 4 + 2 R_max]  result of the y pass (rows ty0-2 .. ty0+33)
//   gs   [36][132]                 G_{o,k} on the tile plus a 2-px halo
//   Ls   [4][34][130]              L_{o,k} on the tile plus a 1-px halo
#include <type_traits>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kRows = kTY + 2 * kHalo;   // 36 rows of G per tile
constexpr int kGP = kTX + 2 * kHalo;     // 132: row pitch of gs
constexpr int kLR = kTY + 2;             // 34 rows of L
constexpr int kLP = kTX + 2;             // 130: row pitch of Ls
constexpr int kStripV = 12;              // outputs per thread in the y pass
constexpr int kStripH = 12;              // outputs per thread in the x pass
static_assert(kRows % kStripV == 0, "y-pass strips must tile the rows");
static_assert(kGP % kStripH == 0, "x-pass strips must tile the columns");
static_assert((kTX * kTY) % kDetThreads == 0, "extremum loop must be warp-uniform");

__device__ __forceinline__ float to_f(uint8_t v) { return (float)v - 128.0f; }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// y pass: tmp[row][c] = sum_d g[|d|] * base[clamp(y + d)][clamp(x)],
// row <-> y = ty0 - 2 + row, c <-> x = tx0 - 2 - R + c.
template <int R, typename InT>
__device__ __forceinline__ void vpass(const InT* __restrict__ src, int spitch, int W, int H,
                                      int tx0, int ty0, const float (&g)[R + 1], float* tmp,
                                      int tpitch) {
  constexpr int kNStrip = kRows / kStripV;
  const int cols = kTX + 2 * kHalo + 2 * R;
  const int xbase = tx0 - kHalo - R;
  const int ybase = ty0 - kHalo - R;
  for (int item = threadIdx.x; item < cols * kNStrip; item += kDetThreads) {
    const int s = item / cols;
    const int c = item - s * cols;
    const int x = min(max(xbase + c, 0), W - 1);
    const InT* col = src + x;
    const int r0 = s * kStripV;
    float acc[kStripV];
#pragma unroll
    for (int o = 0; o < kStripV; ++o) acc[o] = 0.0f;
#pragma unroll
    for (int j = 0; j < kStripV + 2 * R; ++j) {
      const int y = min(max(ybase + r0 + j, 0), H - 1);
      const float v = to_f(col[(size_t)y * spitch]);
#pragma unroll
      for (int o = 0; o < kStripV; ++o) {
        const int d = j - o - R;
        if (d >= -R && d <= R) acc[o] = fmaf(g[d < 0 ? -d : d], v, acc[o]);
      }
    }
#pragma unroll
    for (int o = 0; o < kStripV; ++o) tmp[(r0 + o) * tpitch + c] = acc[o];
  }
}

// x pass: gs[row][c] = sum_d g[|d|] * tmp[row][c + R + d], c <-> x = tx0 - 2 + c.
template <int R>
__device__ __forceinline__ void hpass(const float* tmp, int tpitch, const float (&g)[R + 1],
                                      float* gs) {
  constexpr int kNS = kGP / kStripH;
  for (int item = threadIdx.x; item < kRows * kNS; item += kDetThreads) {
    const int row = item / kNS;
    const int c0 = (item - row * kNS) * kStripH;
    const float* in = tmp + row * tpitch + c0;
    float acc[kStripH];
#pragma unroll
    for (int o = 0; o < kStripH; ++o) acc[o] = 0.0f;
#pragma unroll
    for (int j = 0; j < kStripH + 2 * R; ++j) {
      const float v = in[j];
#pragma unroll
      for (int o = 0; o < kStripH; ++o) {
        const int d = j - o - R;
        if (d >= -R && d <= R) acc[o] = fmaf(g[d < 0 ? -d : d], v, acc[o]);
      }
    }
#pragma unroll
    for (int o = 0; o < kStripH; ++o) gs[row * kGP + c0 + o] = acc[o];
  }
}

template <int R, typename InT>
__device__ __forceinline__ void level_filter(const float* taps, const InT* src, int spitch, int W,
                                             int H, int tx0, int ty0, float* tmp, int tpitch,
                                             float* gs) {
  float g[R + 1];
#pragma unroll
  for (int j = 0; j <= R; ++j) g[j] = taps[j];
  vpass<R, InT>(src, spitch, W, H, tx0, ty0, g, tmp, tpitch);
  __syncthreads();
  hpass<R>(tmp, tpitch, g, gs);
}

template <typename InT>
__device__ void filter_dispatch(int R, const float* taps, const InT* src, int spitch, int W, int H,
                                int tx0, int ty0, float* tmp, int tpitch, float* gs) {
#define CDVS_CASE(r) \
  case r:            \
    level_filter<r, InT>(taps, src, spitch, W, H, tx0, ty0, tmp, tpitch, gs); \
    break;
  switch (R) {
    CDVS_CASE(0) CDVS_CASE(1) CDVS_CASE(2) CDVS_CASE(3) CDVS_CASE(4) CDVS_CASE(5) CDVS_CASE(6)
    CDVS_CASE(7) CDVS_CASE(8) CDVS_CASE(9) CDVS_CASE(10) CDVS_CASE(11) CDVS_CASE(12)
    CDVS_CASE(13) CDVS_CASE(14) CDVS_CASE(15) CDVS_CASE(16) CDVS_CASE(17) CDVS_CASE(18)
    CDVS_CASE(19) CDVS_CASE(20) CDVS_CASE(21) CDVS_CASE(22) CDVS_CASE(23) CDVS_CASE(24)
    default:
      break;  // rejected on the host
  }
#undef CDVS_CASE
}

__device__ __forceinline__ void store4(float* d, const float* s) {
  *reinterpret_cast<float4*>(d) = make_float4(s[0], s[1], s[2], s[3]);
}
__device__ __forceinline__ void store4(__half* d, const float* s) {
  __half2 a = __floats2half2_rn(s[0], s[1]);
  __half2 b = __floats2half2_rn(s[2], s[3]);
  uint2 u;
  u.x = *reinterpret_cast<unsigned*>(&a);
  u.y = *reinterpret_cast<unsigned*>(&b);
  *reinterpret_cast<uint2*>(d) = u;
}
__device__ __forceinline__ void store1(float* d, float v) { *d = v; }
__device__ __forceinline__ void store1(__half* d, float v) { *d = __float2half_rn(v); }

// Tile interior of G_{o,k} -> level storage (4 consecutive x per thread; the
// row pitch is a multiple of 8 elements, so x + 3 < pitch always holds).
template <typename StoreT>
__device__ __forceinline__ void store_level(const float* gs, StoreT* dst, int lpitch, int W, int H,
                                            int tx0, int ty0) {
  constexpr int kQ = kTX / 4;
  for (int i = threadIdx.x; i < kTY * kQ; i += kDetThreads) {
    const int r = i / kQ;
    const int c = (i - r * kQ) * 4;
    const int y = ty0 + r, x = tx0 + c;
    if (y >= H || x >= W) continue;
    const float* s = gs + (r + kHalo) * kGP + c + kHalo;
    float v[4] = {s[0], s[1], s[2], s[3]};
    store4(dst + (size_t)y * lpitch + x, v);
  }
}

// Alg. 1: G_{o+1,0}[i][j] = G_{o,K-1}[2i][2j] for the even pixels of this tile.
template <typename StoreT>
__device__ __forceinline__ void store_decimated(const float* gs, StoreT* dst, int lpitch1, int W,
                                                int H, int tx0, int ty0) {
  constexpr int kHX = kTX / 2, kHY = kTY / 2;
  for (int i = threadIdx.x; i < kHX * kHY; i += kDetThreads) {
    const int r = i / kHX;
    const int c = i - r * kHX;
    const int y = ty0 + 2 * r, x = tx0 + 2 * c;
    if (y >= H || x >= W) continue;
    store1(dst + (size_t)(y >> 1) * lpitch1 + (x >> 1), gs[(2 * r + kHalo) * kGP + 2 * c + kHalo]);
  }
}

template <typename InT, typename StoreT>
__global__ void __launch_bounds__(kDetThreads, 2)
    detect_kernel(const __grid_constant__ DetectArgs a, int tpitch) {
  extern __shared__ float4 smem4[];
  float* tmp = reinterpret_cast<float*>(smem4);
  float* gs = tmp + kRows * tpitch;
  float* Ls = gs + kRows * kGP;

  // (image, tile) of this CTA: largest i with tile_prefix[i] <= blockIdx.x
  const int b = blockIdx.x;
  int lo = 0, hi = a.n_images;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.tile_prefix[mid] <= b) lo = mid;
    else hi = mid;
  }
  const int img = lo;
  const ImgPlan* P = a.plans + img;
  const int o = a.octave;
  const OctPlan op = P->oct[o];
  const int W = op.W, H = op.H, lpitch = op.lpitch;
  const int t = b - a.tile_prefix[img];
  const int tx0 = (t % op.tiles_x) * kTX;
  const int ty0 = (t / op.tiles_x) * kTY;
  StoreT* lev = reinterpret_cast<StoreT*>(a.levels) + op.level_off;
  const size_t lstride = (size_t)lpitch * H;

  const InT* src;
  int spitch;
  if constexpr (std::is_same<InT, uint8_t>::value) {
    src = reinterpret_cast<const InT*>(P->src);
    spitch = P->pitch;
  } else {
    src = reinterpret_cast<const InT*>(lev);  // level (o, 0) is the octave base
    spitch = lpitch;
  }

  for (int k = 0; k < kScales; ++k) {
    filter_dispatch<InT>(a.radius[k], a.taps[k], src, spitch, W, H, tx0, ty0, tmp, tpitch, gs);
    __syncthreads();
    if (k > 0 || a.write_level0) store_level<StoreT>(gs, lev + k * lstride, lpitch, W, H, tx0, ty0);
    if (k == kScales - 1 && o + 1 < P->n_oct) {
      const OctPlan op1 = P->oct[o + 1];
      store_decimated<StoreT>(gs, reinterpret_cast<StoreT*>(a.levels) + op1.level_off, op1.lpitch,
                              W, H, tx0, ty0);
    }
    // L_{o,k} = s_k^2 * 5-point Laplacian, clamp-to-edge at the image border
    const float s2 = a.s2[k];
    float* Lk = Ls + k * (kLR * kLP);
    for (int i = threadIdx.x; i < kLR * kLP; i += kDetThreads) {
      const int ly = i / kLP, lx = i - (i / kLP) * kLP;
      const int y = ty0 - 1 + ly, x = tx0 - 1 + lx;
      float L = 0.0f;
      if (x >= 0 && x < W && y >= 0 && y < H) {
        const int gr = ly + 1, gc = lx + 1;
        const int cl = x > 0 ? gc - 1 : gc, cr = x < W - 1 ? gc + 1 : gc;
        const int ru = y > 0 ? gr - 1 : gr, rd = y < H - 1 ? gr + 1 : gr;
        const float c = gs[gr * kGP + gc];
        L = s2 * ((gs[gr * kGP + cl] + gs[gr * kGP + cr]) + (gs[ru * kGP + gc] + gs[rd * kGP + gc]) -
                  4.0f * c);
      }
      Lk[i] = L;
    }
    __syncthreads();
  }

  // ---- ALP extremum (Eq. 2-3), 8-neighbour test, refinement (stage B)
  const int lane = threadIdx.x & 31;
  Cand* qout = a.cands + (size_t)img * a.cand_cap;
  for (int it = 0; it < (kTX * kTY) / kDetThreads; ++it) {
    const int idx = it * kDetThreads + threadIdx.x;
    const int ly = idx / kTX, lx = idx - (idx / kTX) * kTX;
    const int x = tx0 + lx, y = ty0 + ly;
    bool found = false;
    Cand c;
    if (x >= 1 && x < W - 1 && y >= 1 && y < H - 1) {
      const int li = (ly + 1) * kLP + (lx + 1);
      float L[kScales];
#pragma unroll
      for (int k = 0; k < kScales; ++k) L[k] = Ls[k * (kLR * kLP) + li];
      float al[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kScales; ++k) s = fmaf(a.B[i][k], L[k], s);
        al[i] = s;
      }
      // roots of p'(t) = 3 a3 t^2 + 2 a2 t + a1 in cancellation-free form
      const float A = 3.0f * al[3], Bq = 2.0f * al[2], C = al[1];
      float roots[2];
      int nr = 0;
      if (A == 0.0f) {
        if (Bq != 0.0f) roots[nr++] = -C / Bq;
      } else {
        const float D = Bq * Bq - 4.0f * A * C;
        if (D > 0.0f) {
          const float q = -0.5f * (Bq + copysignf(sqrtf(D), Bq));
          roots[nr++] = q / A;
          if (q != 0.0f) roots[nr++] = C / q;
        }
      }
      int bt = 0;
      float btv = 0.0f, bv = 0.0f;
      for (int r = 0; r < nr; ++r) {
        const float tt = roots[r];
        if (!(tt >= a.t_lo && tt <= a.t_hi)) continue;
        const float pdd = 6.0f * al[3] * tt + 2.0f * al[2];
        if (pdd == 0.0f) continue;
        const float v = ((al[3] * tt + al[2]) * tt + al[1]) * tt + al[0];
        if (!(fabsf(v) >= a.T)) continue;
        if (bt == 0 || fabsf(v) > fabsf(bv) || (fabsf(v) == fabsf(bv) && tt < btv)) {
          bt = pdd < 0.0f ? 1 : -1;
          btv = tt;
          bv = v;
        }
      }
      if (bt != 0) {
        // weights of the K samples in p(t*): w_k = sum_i B[i][k] t*^i
        float w[kScales];
#pragma unroll
        for (int k = 0; k < kScales; ++k)
          w[k] = fmaf(fmaf(fmaf(a.B[3][k], btv, a.B[2][k]), btv, a.B[1][k]), btv, a.B[0][k]);
        float q[9];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const int lj = li + dy * kLP + dx;
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < kScales; ++k) s = fmaf(w[k], Ls[k * (kLR * kLP) + lj], s);
            q[(dy + 1) * 3 + (dx + 1)] = s;
          }
        bool ok = true;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          if (j == 4) continue;
          if (bt > 0 ? !(q[j] < q[4]) : !(q[j] > q[4])) ok = false;
        }
        if (ok) {
          const float gx = 0.5f * (q[5] - q[3]);
          const float gy = 0.5f * (q[7] - q[1]);
          const float hxx = q[5] - 2.0f * q[4] + q[3];
          const float hyy = q[7] - 2.0f * q[4] + q[1];
          const float hxy = 0.25f * (q[8] - q[6] - q[2] + q[0]);
          const float det = hxx * hyy - hxy * hxy;
          if (det > 0.0f) {
            const float tr = hxx + hyy;
            const float ratio = tr * tr / det;
            if (ratio < a.edge_lim) {
              const float ddx = -(hyy * gx - hxy * gy) / det;
              const float ddy = -(hxx * gy - hxy * gx) / det;
              if (fabsf(ddx) <= a.offset_max && fabsf(ddy) <= a.offset_max) {
                const float ph = q[4] + 0.5f * (gx * ddx + gy * ddy);
                if (fabsf(ph) >= a.T) {
                  c.xo = (float)x + ddx;
                  c.yo = (float)y + ddy;
                  c.so = a.tc + btv;
                  c.resp = ph;
                  c.pss = 6.0f * al[3] * btv + 2.0f * al[2];
                  c.ratio = ratio;
                  c.octave = (short)o;
                  c.type = (short)bt;
                  c.spare = 0;
                  found = true;
                }
              }
            }
          }
        }
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, found);
    if (m) {
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(a.cand_count + img, __popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (found) {
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        if (pos < a.cand_cap) qout[pos] = c;
        else atomicOr(a.status, kStatusCandOverflow);
      }
    }
  }
}

}  // namespace

size_t detect_smem_bytes(int max_radius) {
  const int tpitch = kTX + 2 * kHalo + 2 * max_radius;
  return sizeof(float) * ((size_t)kRows * tpitch + (size_t)kRows * kGP + (size_t)kScales * kLR * kLP);
}

cudaError_t launch_detect(const DetectArgs& a, int n_tiles, int max_radius, int storage,
                          cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  const int tpitch = kTX + 2 * kHalo + 2 * max_radius;
  const size_t smem = detect_smem_bytes(max_radius);
  cudaError_t e;
#define CDVS_LAUNCH(IN, ST)                                                                     \
  do {                                                                                          \
    e = cudaFuncSetAttribute(detect_kernel<IN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                        \
    if (e != cudaSuccess) return e;                                                             \
    detect_kernel<IN, ST><<<n_tiles, kDetThreads, smem, s>>>(a, tpitch);                        \
  } while (0)
  if (storage == CDVS_STORAGE_FP16) {
    if (a.octave == 0) CDVS_LAUNCH(uint8_t, __half);
    else CDVS_LAUNCH(__half, __half);
  } else {
    if (a.octave == 0) CDVS_LAUNCH(uint8_t, float);
    else CDVS_LAUNCH(float, float);
  }
#undef CDVS_LAUNCH
  return cudaGetLastError();
}

}  // namespace cdvs
