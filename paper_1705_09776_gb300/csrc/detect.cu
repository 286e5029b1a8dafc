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
// The filters run on packed FP32 pairs (fma.rn.f32x2: two independent
// round-to-nearest FMAs per instruction): the y pass on pairs of adjacent
// columns, the x pass on pairs of adjacent rows.  Intermediate images are kept
// "row-pair interleaved" -- element (y, x) of a band starting at row y0 sits at
// [(y - y0) / 2][x][(y - y0) % 2] -- so that every operand pair is one aligned
// 64-bit shared-memory word.
//
// Shared memory per CTA (FP32), Rm = largest level radius of the octave,
// Cm = 16 (Rm <= 14) or 28 (Rm <= 24):
//   in  [36 + 2 Rm][128 + 2 Cm]   octave base with halo, minus 128 at octave 0
//   tmp [18][128 + 2 Cm][2]       y-pass result, rows ty0-2 .. ty0+33
//   gs  [18][132][2]              G_{o,k}, rows ty0-2 .. ty0+33, cols tx0-2 ..
//   Ls  [4][18][130][2]           L_{o,k}, same rows, cols tx0-1 .. tx0+128
// After the last level, `in` and `tmp` hold the list of pixels that pass the
// scale test (phase 1) for the neighbour test and refinement (phase 2).
#include <type_traits>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kRows = kTY + 2 * kHalo;   // 36 rows of G per tile
constexpr int kRP = kRows / 2;           // 18 row pairs
constexpr int kGC = kTX + 2 * kHalo;     // 132 columns of G
constexpr int kLC = kTX + 2;             // 130 columns of L
constexpr int kSV = 6;                   // rows per thread in the y pass
constexpr int kSH = 6;                   // columns per thread in the x pass
constexpr int kLG = 3;                   // row-pair groups in the Laplacian pass
static_assert(kRows % kSV == 0 && kSV % 2 == 0, "y-pass strips must tile the row pairs");
static_assert(kGC % kSH == 0 && kSH % 2 == 0, "x-pass strips must tile the columns");
static_assert(kRP % kLG == 0, "Laplacian groups must tile the row pairs");
static_assert((kTX * kTY / 2) % kDetThreads == 0, "extremum loop must be warp-uniform");

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ float to_f(uint8_t v) { return (float)v - 128.0f; }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// ---- stage the octave base (with clamp-to-edge) into in[IR][IC]
template <typename InT>
__device__ __forceinline__ void stage_input(const InT* __restrict__ src, int spitch, int W, int H,
                                            int tx0, int ty0, int rm, int cm, float* in) {
  const int IR = kRows + 2 * rm, IC = kTX + 2 * cm;
  const int y0 = ty0 - kHalo - rm, x0 = tx0 - cm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kWarps = kDetThreads / 32;
  const bool interior_x = x0 >= 0 && x0 + IC <= W;
  constexpr int kMaxQ = 2;              // 16-byte row chunks per lane: IC / 4 <= 64
  constexpr int kMaxRows = (kRows + 2 * kMaxRadius + kWarps - 1) / kWarps;
  if constexpr (std::is_same<InT, uint8_t>::value) {
    // four bytes per load where the row start and pitch allow it; every load
    // of the thread is issued before the first conversion
    const bool vec = interior_x && ((spitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(src) & 3) == 0);
    if (vec) {
      const int q = IC / 4;
      uchar4 b[kMaxRows][kMaxQ];
#pragma unroll
      for (int i = 0; i < kMaxRows; ++i) {
        const int r = warp + i * kWarps;
        const int y = min(max(y0 + r, 0), H - 1);
        const uchar4* row = reinterpret_cast<const uchar4*>(src + (size_t)y * spitch + x0);
#pragma unroll
        for (int j = 0; j < kMaxQ; ++j) {
          const int c = lane + 32 * j;
          if (r < IR && c < q) b[i][j] = __ldg(row + c);
        }
      }
#pragma unroll
      for (int i = 0; i < kMaxRows; ++i) {
        const int r = warp + i * kWarps;
#pragma unroll
        for (int j = 0; j < kMaxQ; ++j) {
          const int c = lane + 32 * j;
          if (r < IR && c < q)
            reinterpret_cast<float4*>(in + r * IC)[c] =
                make_float4((float)b[i][j].x - 128.0f, (float)b[i][j].y - 128.0f, (float)b[i][j].z - 128.0f,
                            (float)b[i][j].w - 128.0f);
        }
      }
      return;
    }
  } else if constexpr (std::is_same<InT, float>::value) {
    if (interior_x) {  // rows are 16-byte aligned (pitch multiple of 8, x0 multiple of 4)
      const int q = IC / 4;
      float4 b[kMaxRows][kMaxQ];
#pragma unroll
      for (int i = 0; i < kMaxRows; ++i) {
        const int r = warp + i * kWarps;
        const int y = min(max(y0 + r, 0), H - 1);
        const float4* row = reinterpret_cast<const float4*>(src + (size_t)y * spitch + x0);
#pragma unroll
        for (int j = 0; j < kMaxQ; ++j) {
          const int c = lane + 32 * j;
          if (r < IR && c < q) b[i][j] = __ldg(row + c);
        }
      }
#pragma unroll
      for (int i = 0; i < kMaxRows; ++i) {
        const int r = warp + i * kWarps;
#pragma unroll
        for (int j = 0; j < kMaxQ; ++j) {
          const int c = lane + 32 * j;
          if (r < IR && c < q) reinterpret_cast<float4*>(in + r * IC)[c] = b[i][j];
        }
      }
      return;
    }
  }
  for (int r = warp; r < IR; r += kWarps) {
    const int y = min(max(y0 + r, 0), H - 1);
    const InT* row = src + (size_t)y * spitch;
    for (int c = lane; c < IC; c += 32) in[r * IC + c] = to_f(row[min(max(x0 + c, 0), W - 1)]);
  }
}

// ---- y pass on column pairs: tmp rows ty0-2 .. ty0+33, columns from
// x = tx0 - C (C = 2 + R rounded up to even) to tx0 + 128 + C.
template <int R, int ic>
__device__ __forceinline__ void vpass(const float* in, int rm, int cm, const float2 (&g)[R + 1], float* tmp) {
  constexpr int C = (2 + R + 1) & ~1;
  constexpr int kPairs = (kTX + 2 * C) / 2;
  constexpr int kStrips = kRows / kSV;
  const int col_off = cm - C;  // in-column of tmp column 0
  for (int item = threadIdx.x; item < kPairs * kStrips; item += kDetThreads) {
    const int s = item / kPairs;
    const int p = item - s * kPairs;
    const int r0 = s * kSV;
    // output row r reads in-rows r + rm + d, d in [-R, R]
    const float* src = in + (r0 + rm - R) * ic + col_off + 2 * p;
    float2 acc[kSV];
#pragma unroll
    for (int o = 0; o < kSV; ++o) acc[o] = f2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < kSV + 2 * R; ++j) {
      const float2 v = *reinterpret_cast<const float2*>(src + j * ic);
#pragma unroll
      for (int o = 0; o < kSV; ++o) {
        const int d = j - o - R;
        if (d >= -R && d <= R) acc[o] = fma2(g[d < 0 ? -d : d], v, acc[o]);
      }
    }
    // rows r0+o, r0+o+1 of columns 2p, 2p+1 -> one 16-byte store
    float* dst = tmp + ((size_t)(r0 / 2) * ic + 2 * p) * 2;
#pragma unroll
    for (int o = 0; o < kSV; o += 2)
      *reinterpret_cast<float4*>(dst + (size_t)(o / 2) * ic * 2) =
          make_float4(acc[o].x, acc[o + 1].x, acc[o].y, acc[o + 1].y);
  }
}

// ---- x pass on row pairs: gs[yp][c] (c <-> x = tx0 - 2 + c) from tmp
template <int R, int ic>
__device__ __forceinline__ void hpass(const float* tmp, const float2 (&g)[R + 1], float* gs) {
  constexpr int C = (2 + R + 1) & ~1;
  constexpr int kNS = kGC / kSH;
  constexpr int kOff = C - 2 - R;  // tmp column of output column 0's first tap (0 or 1)
  constexpr int kIn = kSH + 2 * R;
  for (int item = threadIdx.x; item < kRP * kNS; item += kDetThreads) {
    const int yp = item / kNS;
    const int c0 = (item - yp * kNS) * kSH;
    const float2* t = reinterpret_cast<const float2*>(tmp) + (size_t)yp * ic + c0 + kOff;
    float2 acc[kSH];
#pragma unroll
    for (int o = 0; o < kSH; ++o) acc[o] = f2(0.0f, 0.0f);
    if constexpr (kOff == 0) {
      // 16-byte loads: two consecutive columns of the row pair
#pragma unroll
      for (int j = 0; j < kIn; j += 2) {
        const float4 v4 = *reinterpret_cast<const float4*>(t + j);
        const float2 va = f2(v4.x, v4.y), vb = f2(v4.z, v4.w);
#pragma unroll
        for (int o = 0; o < kSH; ++o) {
          const int d = j - o - R;
          if (d >= -R && d <= R) acc[o] = fma2(g[d < 0 ? -d : d], va, acc[o]);
          const int d1 = d + 1;
          if (j + 1 < kIn && d1 >= -R && d1 <= R) acc[o] = fma2(g[d1 < 0 ? -d1 : d1], vb, acc[o]);
        }
      }
    } else {
      // t is 8 bytes past a 16-byte boundary: one 8-byte load, then 16-byte
      // loads, then one 8-byte load (kIn is even)
      float2 v[kIn];
      v[0] = t[0];
#pragma unroll
      for (int j = 1; j + 1 < kIn; j += 2) {
        const float4 v4 = *reinterpret_cast<const float4*>(t + j);
        v[j] = f2(v4.x, v4.y);
        v[j + 1] = f2(v4.z, v4.w);
      }
      v[kIn - 1] = t[kIn - 1];
#pragma unroll
      for (int j = 0; j < kIn; ++j) {
#pragma unroll
        for (int o = 0; o < kSH; ++o) {
          const int d = j - o - R;
          if (d >= -R && d <= R) acc[o] = fma2(g[d < 0 ? -d : d], v[j], acc[o]);
        }
      }
    }
    float4* dst = reinterpret_cast<float4*>(gs + ((size_t)yp * kGC + c0) * 2);
#pragma unroll
    for (int o = 0; o < kSH; o += 2) dst[o / 2] = make_float4(acc[o].x, acc[o].y, acc[o + 1].x, acc[o + 1].y);
  }
}

template <int R, int ic>
__device__ __forceinline__ void level_filter(const float* taps, const float* in, int rm, int cm, float* tmp,
                                             float* gs) {
  float2 g[R + 1];
#pragma unroll
  for (int j = 0; j <= R; ++j) g[j] = f2(taps[j], taps[j]);
  vpass<R, ic>(in, rm, cm, g, tmp);
  __syncthreads();
  hpass<R, ic>(tmp, g, gs);
}

template <int ic>
__device__ void filter_dispatch(int R, const float* taps, const float* in, int rm, int cm, float* tmp,
                                float* gs) {
#define CDVS_CASE(r)                                    \
  case r:                                               \
    if constexpr (2 + r <= (ic - kTX) / 2) level_filter<r, ic>(taps, in, rm, cm, tmp, gs); \
    break;
  switch (R) {
    CDVS_CASE(0) CDVS_CASE(1) CDVS_CASE(2) CDVS_CASE(3) CDVS_CASE(4) CDVS_CASE(5) CDVS_CASE(6)
    CDVS_CASE(7) CDVS_CASE(8) CDVS_CASE(9) CDVS_CASE(10) CDVS_CASE(11) CDVS_CASE(12)
    CDVS_CASE(13) CDVS_CASE(14) CDVS_CASE(15) CDVS_CASE(16) CDVS_CASE(17) CDVS_CASE(18)
    CDVS_CASE(19) CDVS_CASE(20) CDVS_CASE(21) CDVS_CASE(22) CDVS_CASE(23) CDVS_CASE(24)
    default:
      __syncthreads();  // rejected on the host; keep the barrier count uniform
      break;
  }
#undef CDVS_CASE
}

// gs element (row r, col c) of the row-pair layout
__device__ __forceinline__ float& gat(float* gs, int r, int c) { return gs[((r >> 1) * kGC + c) * 2 + (r & 1)]; }

// Clamp-to-edge for the Laplacian: the column and row just outside the
// image take the value of the nearest image pixel, so the stencil below
// needs no border cases (the Laplacian is only used at image pixels).
__device__ __forceinline__ void replicate_borders(float* gs, int W, int H, int tx0, int ty0) {
  const int cl = 1 - tx0;             // gs column of x = -1 (valid when tx0 == 0)
  const int cr = W - tx0 + kHalo;     // gs column of x = W
  const int rt = 1 - ty0, rb = H - ty0 + kHalo;
  const bool left = tx0 == 0, right = cr < kGC, top = ty0 == 0, bottom = rb < kRows;
  if (!(left || right || top || bottom)) return;  // uniform over the CTA
  if (left || right) {
    for (int r = threadIdx.x; r < kRows; r += kDetThreads) {
      if (left) gat(gs, r, cl) = gat(gs, r, cl + 1);
      if (right) gat(gs, r, cr) = gat(gs, r, cr - 1);
    }
    __syncthreads();
  }
  if (top || bottom) {
    for (int c = threadIdx.x; c < kGC; c += kDetThreads) {
      if (top) gat(gs, rt, c) = gat(gs, rt + 1, c);
      if (bottom) gat(gs, rb, c) = gat(gs, rb - 1, c);
    }
    __syncthreads();
  }
}

// L_{o,k} = s_k^2 * (left + right + up + down - 4 centre) on row pairs; each
// thread walks one column down kRP / kLG row pairs with a sliding window.
// (The first and last tile rows of the band get a clamped, unused value.)
__device__ __forceinline__ void laplacian(const float* gs, float s2k, float* L) {
  constexpr int kPer = kRP / kLG;
  const float2 s2 = f2(s2k, s2k), m4 = f2(-4.0f, -4.0f);
  const float2* g = reinterpret_cast<const float2*>(gs);
  float2* out = reinterpret_cast<float2*>(L);
  for (int item = threadIdx.x; item < kLC * kLG; item += kDetThreads) {
    const int grp = item / kLC;
    const int c = item - grp * kLC;  // L column c <-> gs column c + 1
    const int yp0 = grp * kPer;
    float2 up = g[max(yp0 - 1, 0) * kGC + c + 1];
    float2 ce = g[yp0 * kGC + c + 1];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int yp = yp0 + k;
      const float2 dn = g[min(yp + 1, kRP - 1) * kGC + c + 1];
      const float2 le = g[yp * kGC + c], ri = g[yp * kGC + c + 2];
      // rows 2yp, 2yp+1: up neighbours (row 2yp-1, row 2yp), down (row 2yp+1, row 2yp+2)
      const float2 vs = f2(up.y + ce.y, ce.x + dn.x);
      const float2 t = add2(add2(le, ri), vs);
      out[yp * kLC + c] = mul2(s2, fma2(m4, ce, t));
      up = ce;
      ce = dn;
    }
  }
}

__device__ __forceinline__ void store2(float* d, float a, float b) { *reinterpret_cast<float2*>(d) = f2(a, b); }
__device__ __forceinline__ void store2(__half* d, float a, float b) {
  *reinterpret_cast<__half2*>(d) = __floats2half2_rn(a, b);
}
__device__ __forceinline__ void store1(float* d, float v) { *d = v; }
__device__ __forceinline__ void store1(__half* d, float v) { *d = __float2half_rn(v); }

// Tile interior of G_{o,k} -> level storage.  Each thread takes 2 columns of a
// row pair (one 16-byte shared load) and writes 2 x 2 values; the row pitch is
// a multiple of 8 elements, so x + 1 < pitch always holds.
template <typename StoreT>
__device__ __forceinline__ void store_level(const float* gs, StoreT* dst, int lpitch, int W, int H, int tx0,
                                            int ty0) {
  constexpr int kQ = kTX / 2;
  for (int i = threadIdx.x; i < (kTY / 2) * kQ; i += kDetThreads) {
    const int m = i / kQ;                 // tile rows 2m, 2m+1 = gs row pair m + 1
    const int c = (i - m * kQ) * 2;       // tile columns c, c+1 = gs columns c+2, c+3
    const int x = tx0 + c, y = ty0 + 2 * m;
    if (x >= W || y >= H) continue;
    const float4 v = *reinterpret_cast<const float4*>(gs + ((m + 1) * kGC + c + kHalo) * 2);
    store2(dst + (size_t)y * lpitch + x, v.x, v.z);
    if (y + 1 < H) store2(dst + (size_t)(y + 1) * lpitch + x, v.y, v.w);
  }
}

// Alg. 1: G_{o+1,0}[i][j] = G_{o,K-1}[2i][2j] for the even pixels of this tile.
template <typename StoreT>
__device__ __forceinline__ void store_decimated(const float* gs, StoreT* dst, int lpitch1, int W, int H,
                                                int tx0, int ty0) {
  constexpr int kHX = kTX / 2, kHY = kTY / 2;
  for (int i = threadIdx.x; i < kHX * kHY; i += kDetThreads) {
    const int r = i / kHX;
    const int c = i - r * kHX;
    const int y = ty0 + 2 * r, x = tx0 + 2 * c;
    if (y >= H || x >= W) continue;
    // tile row 2r is the first row of gs pair r + 1; 16-byte load of columns 2c+2, 2c+3
    const float4 v = *reinterpret_cast<const float4*>(gs + ((r + 1) * kGC + 2 * c + kHalo) * 2);
    store1(dst + (size_t)(y >> 1) * lpitch1 + (x >> 1), v.x);
  }
}

struct Found {
  float xo, yo, so, resp, pss, ratio;
  int type;
};

__device__ __forceinline__ float2 abs2(float2 v) { return f2(fabsf(v.x), fabsf(v.y)); }
__device__ __forceinline__ float2 rcp2(float2 v) { return f2(__frcp_rn(v.x), __frcp_rn(v.y)); }

// S4 on a pair of pixels (phase 1): for each pixel, the admissible extremum
// of the cubic p(t) = a0 + a1 t + a2 t^2 + a3 t^3 with |p| >= T.  The roots of
// p'(t) = 3 a3 t^2 + 2 a2 t + a1 come from the cancellation-free form
// q = -(B + sign(B) sqrt(D)) / 2, t = q / A and C / q; when both are admissible
// the larger |p| wins (ties: the smaller t).  bt = +1 maximum, -1 minimum, 0.
__device__ __forceinline__ void cubic_extremum2(const DetectArgs& a, const float2 (&al)[4], bool live0,
                                                bool live1, int (&bt)[2], float (&tb)[2]) {
  bt[0] = bt[1] = 0;
  tb[0] = tb[1] = 0.0f;
  // no t in [t_lo, t_hi] can reach |p| >= T when this bound is below T
  const float mm = fmaxf(-a.t_lo, a.t_hi);
  const float2 m2 = f2(mm, mm);
  const float2 bound = add2(abs2(al[0]), mul2(m2, add2(abs2(al[1]), mul2(m2, fma2(m2, abs2(al[3]), abs2(al[2]))))));
  const float Tb = a.T * 0.99999f;
  const bool go0 = live0 && bound.x >= Tb, go1 = live1 && bound.y >= Tb;
  if (!(go0 || go1)) return;
  const float2 A = mul2(f2(3.0f, 3.0f), al[3]), Bq = mul2(f2(2.0f, 2.0f), al[2]), C = al[1];
  const float2 D = fma2(mul2(f2(-4.0f, -4.0f), A), C, mul2(Bq, Bq));
  const float2 sq = f2(sqrtf(fmaxf(D.x, 0.0f)), sqrtf(fmaxf(D.y, 0.0f)));
  const float2 q = mul2(f2(-0.5f, -0.5f), add2(Bq, f2(copysignf(sq.x, Bq.x), copysignf(sq.y, Bq.y))));
  const float2 r0 = mul2(q, rcp2(A));
  const float2 r1 = mul2(C, rcp2(q));
  const float2 six_a3 = mul2(f2(6.0f, 6.0f), al[3]);
  const float2 two_a2 = mul2(f2(2.0f, 2.0f), al[2]);
  // p'' and p at both roots, both pixels
  const float2 pdd0 = fma2(six_a3, r0, two_a2), pdd1 = fma2(six_a3, r1, two_a2);
  const float2 v0 = fma2(fma2(fma2(al[3], r0, al[2]), r0, al[1]), r0, al[0]);
  const float2 v1 = fma2(fma2(fma2(al[3], r1, al[2]), r1, al[1]), r1, al[0]);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!(h ? go1 : go0)) continue;
    const float Ah = h ? A.y : A.x, Bh = h ? Bq.y : Bq.x, Ch = h ? C.y : C.x;
    const float Dh = h ? D.y : D.x, qh = h ? q.y : q.x;
    float t0, t1, p0, p1, s0, s1;
    int nr;
    if (Ah == 0.0f) {  // quadratic p: the single root of the linear derivative
      if (Bh == 0.0f) continue;
      t0 = -Ch / Bh;
      s0 = h ? two_a2.y : two_a2.x;
      p0 = h ? fmaf(fmaf(fmaf(al[3].y, t0, al[2].y), t0, al[1].y), t0, al[0].y)
             : fmaf(fmaf(fmaf(al[3].x, t0, al[2].x), t0, al[1].x), t0, al[0].x);
      t1 = p1 = s1 = 0.0f;
      nr = 1;
    } else {
      if (!(Dh > 0.0f)) continue;
      t0 = h ? r0.y : r0.x;
      p0 = h ? v0.y : v0.x;
      s0 = h ? pdd0.y : pdd0.x;
      t1 = h ? r1.y : r1.x;
      p1 = h ? v1.y : v1.x;
      s1 = h ? pdd1.y : pdd1.x;
      nr = qh != 0.0f ? 2 : 1;
    }
    int best = 0;
    float bt_t = 0.0f, bv = 0.0f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (r >= nr) break;
      const float tt = r ? t1 : t0, v = r ? p1 : p0, pdd = r ? s1 : s0;
      if (!(tt >= a.t_lo && tt <= a.t_hi)) continue;
      if (pdd == 0.0f) continue;
      if (!(fabsf(v) >= a.T)) continue;
      if (best == 0 || fabsf(v) > fabsf(bv) || (fabsf(v) == fabsf(bv) && tt < bt_t)) {
        best = pdd < 0.0f ? 1 : -1;
        bt_t = tt;
        bv = v;
      }
    }
    bt[h] = best;
    tb[h] = bt_t;
  }
}

// 8-neighbour test at the centre's t* and refinement (Alg. 1 stage B) for
// a pixel that passed phase 1 (phase 2).
__device__ __forceinline__ bool refine_pixel(const DetectArgs& a, const float* Ls, int ly, int lx, int bt,
                                             float btv, int x, int y, Found& f) {
  // weights of the K samples in p(t*): w_k = sum_i B[i][k] t*^i
  float w[kScales];
#pragma unroll
  for (int k = 0; k < kScales; ++k)
    w[k] = fmaf(fmaf(fmaf(a.B[3][k], btv, a.B[2][k]), btv, a.B[1][k]), btv, a.B[0][k]);
  // one address per neighbour row; level and column offsets are constants
  constexpr int kLevel = kRP * kLC * 2;
  float q[9], Lc[kScales];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    const int r = ly + kHalo + dy;
    const float* row = Ls + ((r >> 1) * kLC + lx + 1) * 2 + (r & 1);
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < kScales; ++k) {
        const float L = row[k * kLevel + 2 * dx];
        if (dx == 0 && dy == 0) Lc[k] = L;
        s = fmaf(w[k], L, s);
      }
      q[(dy + 1) * 3 + (dx + 1)] = s;
    }
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    if (j == 4) continue;
    if (bt > 0 ? !(q[j] < q[4]) : !(q[j] > q[4])) return false;
  }
  const float gx = 0.5f * (q[5] - q[3]);
  const float gy = 0.5f * (q[7] - q[1]);
  const float hxx = q[5] - 2.0f * q[4] + q[3];
  const float hyy = q[7] - 2.0f * q[4] + q[1];
  const float hxy = 0.25f * (q[8] - q[6] - q[2] + q[0]);
  const float det = hxx * hyy - hxy * hxy;
  if (!(det > 0.0f)) return false;
  const float tr = hxx + hyy;
  const float ratio = tr * tr / det;
  if (!(ratio < a.edge_lim)) return false;
  const float ddx = -(hyy * gx - hxy * gy) / det;
  const float ddy = -(hxx * gy - hxy * gx) / det;
  if (!(fabsf(ddx) <= a.offset_max && fabsf(ddy) <= a.offset_max)) return false;
  const float ph = q[4] + 0.5f * (gx * ddx + gy * ddy);
  if (!(fabsf(ph) >= a.T)) return false;
  // p''(t*) = 6 a3 t* + 2 a2 from the centre's samples
  float a2 = 0.0f, a3 = 0.0f;
#pragma unroll
  for (int k = 0; k < kScales; ++k) {
    a2 = fmaf(a.B[2][k], Lc[k], a2);
    a3 = fmaf(a.B[3][k], Lc[k], a3);
  }
  f.xo = (float)x + ddx;
  f.yo = (float)y + ddy;
  f.so = a.tc + btv;
  f.resp = ph;
  f.pss = 6.0f * a3 * btv + 2.0f * a2;
  f.ratio = ratio;
  f.type = bt;
  return true;
}

// warp-aggregated append to the image's candidate queue (all lanes call it)
__device__ __forceinline__ void append(const DetectArgs& a, int img, int o, bool found, const Found& f) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, found);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(a.cand_count + img, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (!found) return;
  const int pos = base + __popc(m & ((1u << lane) - 1u));
  if (pos >= a.cand_cap) {
    atomicOr(a.status, kStatusCandOverflow);
    return;
  }
  Cand c;
  c.xo = f.xo;
  c.yo = f.yo;
  c.so = f.so;
  c.resp = f.resp;
  c.pss = f.pss;
  c.ratio = f.ratio;
  c.octave = (short)o;
  c.type = (short)f.type;
  c.spare = 0;
  a.cands[(size_t)img * a.cand_cap + pos] = c;
}

// Phase-1 survivors of a tile: packed (ly, lx, type) and t*.
struct Pending {
  int code;  // ly << 16 | lx << 1 | (type > 0)
  float t;
};

template <typename InT, typename StoreT, int ic>
__global__ void __launch_bounds__(kDetThreads, 1) detect_kernel(const __grid_constant__ DetectArgs a, int rm) {
  extern __shared__ float4 smem4[];
  __shared__ int n_pending;
  const int cm = (ic - kTX) / 2;
  float* in = reinterpret_cast<float*>(smem4);
  float* tmp = in + (kRows + 2 * rm) * ic;
  float* gs = tmp + kRows * ic;
  float* Ls = gs + kRows * kGC;

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

  if constexpr (std::is_same<InT, uint8_t>::value)
    stage_input<InT>(reinterpret_cast<const InT*>(P->src), P->pitch, W, H, tx0, ty0, rm, cm, in);
  else
    stage_input<InT>(reinterpret_cast<const InT*>(lev), lpitch, W, H, tx0, ty0, rm, cm, in);
  if (threadIdx.x == 0) n_pending = 0;
  __syncthreads();

  for (int k = 0; k < kScales; ++k) {
    filter_dispatch<ic>(a.radius[k], a.taps[k], in, rm, cm, tmp, gs);
    __syncthreads();
    replicate_borders(gs, W, H, tx0, ty0);
    if (k > 0 || a.write_level0) store_level<StoreT>(gs, lev + k * lstride, lpitch, W, H, tx0, ty0);
    if (k == kScales - 1 && o + 1 < P->n_oct) {
      const OctPlan op1 = P->oct[o + 1];
      store_decimated<StoreT>(gs, reinterpret_cast<StoreT*>(a.levels) + op1.level_off, op1.lpitch, W, H, tx0,
                              ty0);
    }
    laplacian(gs, a.s2[k], Ls + (size_t)k * kRP * kLC * 2);
    __syncthreads();
  }

  // ---- phase 1, per pixel pair (tile rows 2m, 2m+1 are L row pair m + 1):
  // cubic coefficients of Eq. 3 on packed pairs, then the admissible
  // extremum in scale; survivors are compacted into `in` (no longer needed)
  Pending* pend = reinterpret_cast<Pending*>(in);
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < (kTX * kTY / 2) / kDetThreads; ++it) {
    const int idx = it * kDetThreads + threadIdx.x;
    const int m = idx / kTX, lx = idx - (idx / kTX) * kTX;
    float2 Lk[kScales];
#pragma unroll
    for (int k = 0; k < kScales; ++k) Lk[k] = reinterpret_cast<const float2*>(Ls)[(k * kRP + m + 1) * kLC + lx + 1];
    float2 al2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 s = f2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < kScales; ++k) s = fma2(f2(a.B[i][k], a.B[i][k]), Lk[k], s);
      al2[i] = s;
    }
    const int x = tx0 + lx, y0 = ty0 + 2 * m;
    const bool inx = x >= 1 && x < W - 1;
    int bt[2];
    float tb[2];
    cubic_extremum2(a, al2, inx && y0 >= 1 && y0 < H - 1, inx && y0 + 1 >= 1 && y0 + 1 < H - 1, bt, tb);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned msk = __ballot_sync(0xffffffffu, bt[h] != 0);
      if (msk) {
        const int leader = __ffs(msk) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&n_pending, __popc(msk));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (bt[h] != 0) {
          Pending e;
          e.code = ((2 * m + h) << 16) | (lx << 1) | (bt[h] > 0 ? 1 : 0);
          e.t = tb[h];
          pend[base + __popc(msk & ((1u << lane) - 1u))] = e;
        }
      }
    }
  }
  __syncthreads();

  // ---- phase 2: neighbour test and refinement of the survivors, densely
  const int np = n_pending;
  const int rounds = (np + kDetThreads - 1) / kDetThreads;
  for (int r = 0; r < rounds; ++r) {
    const int i = r * kDetThreads + threadIdx.x;
    Found f;
    bool found = false;
    if (i < np) {
      const Pending e = pend[i];
      const int ly = e.code >> 16, lx = (e.code >> 1) & 0x7fff;
      found = refine_pixel(a, Ls, ly, lx, (e.code & 1) ? 1 : -1, e.t, tx0 + lx, ty0 + ly, f);
    }
    append(a, img, o, found, f);
  }
}

}  // namespace

// The input tile pitch: 128 + 2 Cm columns for radii up to 14 and up to 24.
static int tile_pitch(int max_radius) { return max_radius <= 14 ? 160 : 184; }

size_t detect_smem_bytes(int max_radius) {
  const int ic = tile_pitch(max_radius);
  return sizeof(float) * ((size_t)(kRows + 2 * max_radius) * ic + (size_t)kRows * ic + (size_t)kRows * kGC +
                          (size_t)kScales * kRows * kLC);
}

cudaError_t launch_detect(const DetectArgs& a, int n_tiles, int max_radius, int storage, cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  if (max_radius > kMaxRadius) return cudaErrorInvalidValue;
  const size_t smem = detect_smem_bytes(max_radius);
  cudaError_t e;
#define CDVS_LAUNCH(IN, ST, IC)                                                                                   \
  do {                                                                                                            \
    e = cudaFuncSetAttribute(detect_kernel<IN, ST, IC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                               \
    detect_kernel<IN, ST, IC><<<n_tiles, kDetThreads, smem, s>>>(a, max_radius);                                  \
  } while (0)
#define CDVS_LAUNCH_IC(IN, ST)                                  \
  do {                                                          \
    if (tile_pitch(max_radius) == 160) CDVS_LAUNCH(IN, ST, 160); \
    else CDVS_LAUNCH(IN, ST, 184);                              \
  } while (0)
  if (storage == CDVS_STORAGE_FP16) {
    if (a.octave == 0) CDVS_LAUNCH_IC(uint8_t, __half);
    else CDVS_LAUNCH_IC(__half, __half);
  } else {
    if (a.octave == 0) CDVS_LAUNCH_IC(uint8_t, float);
    else CDVS_LAUNCH_IC(float, float);
  }
#undef CDVS_LAUNCH_IC
#undef CDVS_LAUNCH
  return cudaGetLastError();
}

}  // namespace cdvs
