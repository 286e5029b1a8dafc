// detect_kernel.cuh -- K1, shared by detect.cu (the plain variants) and
// detect_masked.cu (the variants under a block proposal): one octave of interest point detection for a batch of
// images.  A persistent CTA per SM walks over 128x32 output tiles; for each
// tile it computes, fused in shared memory:
//   Gaussian levels G_{o,k} (Eq. 1, Alg. 1 stage A: a pass along y then a
//   pass along x, every level filtered directly from the octave base),
//   scale-normalised 5-point LoG L_{o,k}, the per-pixel cubic in sigma of
//   Eq. 2-3, its extremum scale, the 8-neighbour test, the sub-pixel
//   refinement of Alg. 1 stage B, and appends to the image's candidate queue.
// The same CTA stores its tile of every level (for description) and, on the
// top level, the decimated base of the next octave (Alg. 1: Downsampling
// G_{o,K-1} to G_{o+1,0}).
//
// An octave past the first may be stored transposed, when its transposed
// frame takes fewer tiles (a 320 x 240 octave: 20 tiles instead of 24).  The
// filters are separable and the detector symmetric in x and y, so the kernel
// works in the stored frame unchanged, swaps x and y of the candidates it
// emits, and writes the next octave's base in that octave's orientation.
//
// While a tile is processed, the rows of the next tile's input are already
// on their way into shared memory through asynchronous 16-byte copies
// (cp.async), issued by all threads at once, so global-memory latency overlaps
// the arithmetic.
//
// The filters run on packed FP32 pairs (fma.rn.f32x2: two independent
// round-to-nearest FMAs per instruction): the y pass on pairs of adjacent
// columns, the x pass on pairs of adjacent rows.  Intermediate images are kept
// "row-pair interleaved" -- element (y, x) of a band starting at row y0 sits at
// [(y - y0) / 2][x][(y - y0) % 2] -- so every operand pair is one aligned
// 64-bit shared-memory word.
//
// Shared memory per CTA, Rm = largest level radius of the octave (<= 14 or
// <= 24), IC = 160 or 184 columns, IR = 36 + 2 Rm rows:
//   raw [IR][IC]            next tile's input as stored (u8 or FP32 / FP16)
//   in  [IR][IC]            this tile's input in FP32 (minus 128 at octave 0)
//   tmp [18][IC][2]         y-pass result, rows ty0-2 .. ty0+33
//   gs  [18][132][2]        G_{o,k}, rows ty0-2 .. ty0+33, cols tx0-2 ..
//   Ls  [4][18][130][2]     L_{o,k}, same rows, cols tx0-1 .. tx0+128
// After the last level, `in` and `tmp` hold the list of pixels that pass the
// scale test (phase 1) for the neighbour test and refinement (phase 2).
#pragma once
#include <type_traits>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kGC = kTX + 2 * kHalo;     // 132 columns of G
constexpr int kLC = kTX + 2;             // 130 columns of L

// The work shape of a K1 variant: output tile rows TY (the tile is always 128
// wide), threads per CTA, CTAs per SM the launch bounds ask for, rows per
// thread in the y pass (SV), columns per thread in the x pass (SH), row-pair
// groups in the Laplacian (LG), and whether FP32 input is copied straight
// into the FP32 tile (no staging buffer: the next tile's copies are issued
// once the last y pass has read the current one).
template <int TY_, int THREADS_, int MINB_, int SV_, int SH_, int LG_>
struct Shape {
  static constexpr int TY = TY_, THREADS = THREADS_, MINB = MINB_, SV = SV_, SH = SH_, LG = LG_;
  static constexpr int ROWS = TY + 2 * kHalo;  // rows of G per tile
  static constexpr int RP = ROWS / 2;          // row pairs
  static constexpr int WARPS = THREADS / 32;
  static_assert(ROWS % SV == 0 && SV % 2 == 0, "y-pass strips must tile the row pairs");
  static_assert(kGC % SH == 0 && SH % 2 == 0, "x-pass strips must tile the columns");
  static_assert(RP % LG == 0, "Laplacian groups must tile the row pairs");
  static_assert((kTX * TY / 2) % THREADS == 0, "extremum loop must be warp-uniform");
};

// The variants (index = kernel variant id of the launchers and the tuner):
// one 512-thread CTA per SM on 128 x 32 tiles (y pass 6 or 12 rows per
// thread), or two 256-thread CTAs per SM on 128 x 16 tiles (y pass 4 or 10).
using ShapeA = Shape<32, 512, 1, 6, 6, 3>;
using ShapeB = Shape<32, 512, 1, 12, 6, 3>;
using ShapeC = Shape<16, 256, 2, 4, 6, 2>;
using ShapeD = Shape<16, 256, 2, 10, 6, 2>;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ float to_f(uint8_t v) { return (float)v - 128.0f; }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// ------------------------------------------------ asynchronous copies
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// 16 bytes global -> shared, cached in L2 only; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// this thread's copies have landed (a wait on its own loads, like any load)
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------ tile geometry
// Everything the CTA needs to know about one tile, computed ahead of time by a
// single thread and kept in shared memory.
struct TileInfo {
  long long level_off;  // element offset of level (o, 0) of the tile's image
  long long dec_off;    // level (o + 1, 0), or -1 when o is the image's last octave
  const void* base;     // first input row (u8 image or level (o, 0))
  int img, tx0, ty0;
  int W, H, lpitch;     // octave size and row pitch (elements), stored frame
  int tr;               // the octave is stored transposed (x and y of the frame swapped)
  int dec_tr;           // level (o + 1, 0) is stored in the other orientation
  int dec_pitch;        // row pitch of level (o + 1, 0)
  int pitch;            // input row pitch (elements)
  int cs, ce;           // copied input columns [cs, ce) (image x)
  int bulk;             // rows can be fetched by 16-byte asynchronous copies
  int valid;            // 0 past the launch's last tile
};

// Tile b of the launch (prefix: the launch's tile_prefix, n_images + 1 entries,
// in shared memory): its image is the largest i with prefix[i] <= b.  The
// rows can be copied in 16-byte pieces when source rows, lengths and
// destination rows in raw all start on 16-byte boundaries; otherwise they are
// loaded element by element.
template <typename S, typename InT>
__device__ __noinline__ void tile_info(const DetectArgs& a, const int* prefix, int b, int n_tiles, int ic, TileInfo* out) {
  TileInfo t;
  t.valid = b < n_tiles;
  if (!t.valid) {
    t.bulk = 0;
    *out = t;
    return;
  }
  int lo = 0, hi = a.n_images;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= b) lo = mid;
    else hi = mid;
  }
  const ImgPlan* P = a.plans + lo;
  const OctPlan& op = P->oct[a.octave];
  const int k = b - prefix[lo];
  t.img = lo;
  t.tx0 = (k % op.tiles_x) * kTX;
  t.ty0 = (k / op.tiles_x) * S::TY;
  t.W = op.W;
  t.H = op.H;
  t.lpitch = op.lpitch;
  t.tr = op.tr;
  t.level_off = op.level_off;
  if (a.octave + 1 < P->n_oct) {
    t.dec_off = P->oct[a.octave + 1].level_off;
    t.dec_pitch = P->oct[a.octave + 1].lpitch;
    t.dec_tr = P->oct[a.octave + 1].tr != op.tr;
  } else {
    t.dec_off = -1;
    t.dec_pitch = 0;
    t.dec_tr = 0;
  }
  if constexpr (std::is_same<InT, uint8_t>::value) {
    t.base = P->src;
    t.pitch = P->pitch;
  } else {
    t.base = reinterpret_cast<const InT*>(a.levels) + t.level_off;
    t.pitch = t.lpitch;
  }
  const int cm = (ic - kTX) / 2;
  const int x0 = t.tx0 - cm;
  t.cs = max(x0, 0);
  t.ce = min(x0 + ic, t.W);
  constexpr int es = sizeof(InT);
  t.bulk = ((reinterpret_cast<uintptr_t>(t.base) & 15) == 0) && (((size_t)t.pitch * es) % 16 == 0) &&
           ((t.cs * es) % 16 == 0) && (((t.ce - t.cs) * es) % 16 == 0) && t.ce > t.cs &&
           ((ic * es) % 16 == 0) && (((t.cs - x0) * es) % 16 == 0);
  *out = t;
}

// All threads of the CTA issue the 16-byte copies of every input row of tile
// t into raw (column c of a raw row is image x = tx0 - cm + c; rows clamp to
// the image) and commit them as one group.
template <typename S, typename InT>
__device__ __forceinline__ void issue_tile_copy(const TileInfo& t, int ic, int rm, InT* raw) {
  constexpr int per = 16 / sizeof(InT);  // elements per piece
  const int cm = (ic - kTX) / 2;
  const int IR = S::ROWS + 2 * rm;
  const int y0 = t.ty0 - kHalo - rm;
  const int x0 = t.tx0 - cm;
  const int nc = (t.ce - t.cs) / per;  // pieces per row
  const InT* src = static_cast<const InT*>(t.base) + t.cs;
  InT* dst = raw + (t.cs - x0);
  for (int i = threadIdx.x; i < IR * nc; i += S::THREADS) {
    const int row = i / nc, c = i - row * nc;
    const int y = min(max(y0 + row, 0), t.H - 1);
    cp_async16(dst + (size_t)row * ic + c * per, src + (size_t)y * t.pitch + c * per);
  }
  cp_async_commit();
}

// raw (copied columns only) -> in (FP32), replicating the edge columns.
template <typename S, typename InT>
__device__ __forceinline__ void convert_raw(const InT* raw, const TileInfo& t, int ic, int rm, float* in) {
  const int cm = (ic - kTX) / 2;
  const int IR = S::ROWS + 2 * rm;
  const int x0 = t.tx0 - cm;
  const int clo = t.cs - x0, chi = t.ce - 1 - x0;  // first / last copied column
  const int n4 = ic / 4;
  for (int i = threadIdx.x; i < IR * n4; i += S::THREADS) {
    const int row = i / n4;
    const int c = (i - row * n4) * 4;
    const InT* src = raw + (size_t)row * ic;
    float4 v;
    if (c >= clo && c + 3 <= chi) {
      if constexpr (std::is_same<InT, uint8_t>::value) {
        const uchar4 b = *reinterpret_cast<const uchar4*>(src + c);
        v = make_float4((float)b.x - 128.0f, (float)b.y - 128.0f, (float)b.z - 128.0f, (float)b.w - 128.0f);
      } else if constexpr (std::is_same<InT, float>::value) {
        v = *reinterpret_cast<const float4*>(src + c);
      } else {
        v = make_float4(to_f(src[c]), to_f(src[c + 1]), to_f(src[c + 2]), to_f(src[c + 3]));
      }
    } else {
      v = make_float4(to_f(src[min(max(c, clo), chi)]), to_f(src[min(max(c + 1, clo), chi)]),
                      to_f(src[min(max(c + 2, clo), chi)]), to_f(src[min(max(c + 3, clo), chi)]));
    }
    reinterpret_cast<float4*>(in + (size_t)row * ic)[c / 4] = v;
  }
}

// Element-by-element input load with clamp-to-edge (tiles whose rows cannot
// be copied in 16-byte pieces).
template <typename S, typename InT>
__device__ __forceinline__ void load_tile_direct(const TileInfo& t, int ic, int rm, float* in) {
  const int cm = (ic - kTX) / 2;
  const int IR = S::ROWS + 2 * rm;
  const int y0 = t.ty0 - kHalo - rm, x0 = t.tx0 - cm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int row = warp; row < IR; row += S::WARPS) {
    const int y = min(max(y0 + row, 0), t.H - 1);
    const InT* src = static_cast<const InT*>(t.base) + (size_t)y * t.pitch;
    for (int c = lane; c < ic; c += 32) in[row * ic + c] = to_f(src[min(max(x0 + c, 0), t.W - 1)]);
  }
}

// FP32 rows copied straight into `in` (copied columns only): the columns
// outside the image take the value of the nearest copied one.  Only tiles on
// the left or right image edge have any.
template <typename S>
__device__ __forceinline__ void replicate_in_place(const TileInfo& t, int ic, int rm, float* in) {
  const int cm = (ic - kTX) / 2;
  const int IR = S::ROWS + 2 * rm;
  const int x0 = t.tx0 - cm;
  const int clo = t.cs - x0, chi = t.ce - 1 - x0;
  const int nl = clo, nr = ic - 1 - chi, per = nl + nr;
  if (per == 0) return;
  for (int i = threadIdx.x; i < IR * per; i += S::THREADS) {
    const int row = i / per, c = i - row * per;
    float* r = in + (size_t)row * ic;
    if (c < nl) r[c] = r[clo];
    else r[chi + 1 + (c - nl)] = r[chi];
  }
}

// ------------------------------------------------ separable filters
// y pass on column pairs: tmp rows ty0-2 .. ty0+TY+1, columns from
// x = tx0 - C (C = 2 + R rounded up to even) to tx0 + 128 + C.
template <typename S, int R, int ic>
__device__ __forceinline__ void vpass(const float2* taps, const float* in, int rm, float* tmp) {
  constexpr int kSV = S::SV;
  constexpr int C = (2 + R + 1) & ~1;
  constexpr int kPairs = (kTX + 2 * C) / 2;
  constexpr int kStrips = S::ROWS / kSV;
  constexpr int cm = (ic - kTX) / 2;
  constexpr int col_off = cm - C;  // in-column of tmp column 0
  float2 g[R + 1];
#pragma unroll
  for (int j = 0; j <= R; ++j) g[j] = taps[j];
  for (int item = threadIdx.x; item < kPairs * kStrips; item += S::THREADS) {
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

// x pass on row pairs: gs[yp][c] (c <-> x = tx0 - 2 + c) from tmp
template <typename S, int R, int ic>
__device__ __forceinline__ void hpass(const float2* taps, const float* tmp, float* gs) {
  constexpr int kSH = S::SH, kRP = S::RP;
  constexpr int C = (2 + R + 1) & ~1;
  constexpr int kNS = kGC / kSH;
  constexpr int kOff = C - 2 - R;   // tmp column of output column 0's first tap (0 or 1)
  constexpr int kIn = kSH + 2 * R;  // even
  float2 g[R + 1];
#pragma unroll
  for (int j = 0; j <= R; ++j) g[j] = taps[j];
  for (int item = threadIdx.x; item < kRP * kNS; item += S::THREADS) {
    const int yp = item / kNS;
    const int c0 = (item - yp * kNS) * kSH;
    const float2* t = reinterpret_cast<const float2*>(tmp) + (size_t)yp * ic + c0 + kOff;
    float2 acc[kSH];
#pragma unroll
    for (int o = 0; o < kSH; ++o) acc[o] = f2(0.0f, 0.0f);
    // 16-byte loads (two consecutive columns of the row pair); with kOff = 1
    // the first and the last column come from 8-byte loads
#pragma unroll
    for (int j = 0; j < kIn; j += 2) {
      float2 va, vb;
      if constexpr (kOff == 0) {
        const float4 v4 = *reinterpret_cast<const float4*>(t + j);
        va = f2(v4.x, v4.y);
        vb = f2(v4.z, v4.w);
      } else {
        if (j == 0) {
          va = t[0];
        } else {
          const float4 v4 = *reinterpret_cast<const float4*>(t + j - 1);
          va = f2(v4.z, v4.w);
        }
        if (j + 1 == kIn - 1) {
          vb = t[j + 1];
        } else {
          const float4 v4 = *reinterpret_cast<const float4*>(t + j + 1);
          vb = f2(v4.x, v4.y);
        }
      }
#pragma unroll
      for (int o = 0; o < kSH; ++o) {
        const int d = j - o - R;
        if (d >= -R && d <= R) acc[o] = fma2(g[d < 0 ? -d : d], va, acc[o]);
        const int d1 = d + 1;
        if (d1 >= -R && d1 <= R) acc[o] = fma2(g[d1 < 0 ? -d1 : d1], vb, acc[o]);
      }
    }
    float4* dst = reinterpret_cast<float4*>(gs + ((size_t)yp * kGC + c0) * 2);
#pragma unroll
    for (int o = 0; o < kSH; o += 2) dst[o / 2] = make_float4(acc[o].x, acc[o].y, acc[o + 1].x, acc[o + 1].y);
  }
}

#define CDVS_RC(N, ...) \
  case N: {             \
    constexpr int r = N; \
    __VA_ARGS__;        \
  } break;
#define CDVS_RADIUS_SWITCH(R, ...)                                                                       \
  switch (R) {                                                                                           \
    CDVS_RC(0, __VA_ARGS__) CDVS_RC(1, __VA_ARGS__) CDVS_RC(2, __VA_ARGS__) CDVS_RC(3, __VA_ARGS__)      \
    CDVS_RC(4, __VA_ARGS__) CDVS_RC(5, __VA_ARGS__) CDVS_RC(6, __VA_ARGS__) CDVS_RC(7, __VA_ARGS__)      \
    CDVS_RC(8, __VA_ARGS__) CDVS_RC(9, __VA_ARGS__) CDVS_RC(10, __VA_ARGS__) CDVS_RC(11, __VA_ARGS__)    \
    CDVS_RC(12, __VA_ARGS__) CDVS_RC(13, __VA_ARGS__) CDVS_RC(14, __VA_ARGS__) CDVS_RC(15, __VA_ARGS__)  \
    CDVS_RC(16, __VA_ARGS__) CDVS_RC(17, __VA_ARGS__) CDVS_RC(18, __VA_ARGS__) CDVS_RC(19, __VA_ARGS__)  \
    CDVS_RC(20, __VA_ARGS__) CDVS_RC(21, __VA_ARGS__) CDVS_RC(22, __VA_ARGS__) CDVS_RC(23, __VA_ARGS__)  \
    CDVS_RC(24, __VA_ARGS__)                                                                             \
    default:                                                                                             \
      break;                                                                                             \
  }

template <typename S, int ic>
__device__ void vpass_dispatch(int R, const float2* taps, const float* in, int rm, float* tmp) {
  CDVS_RADIUS_SWITCH(R, if constexpr (2 + r <= (ic - kTX) / 2) vpass<S, r, ic>(taps, in, rm, tmp))
}
template <typename S, int ic>
__device__ void hpass_dispatch(int R, const float2* taps, const float* tmp, float* gs) {
  CDVS_RADIUS_SWITCH(R, if constexpr (2 + r <= (ic - kTX) / 2) hpass<S, r, ic>(taps, tmp, gs))
}

// gs element (row r, col c) of the row-pair layout
__device__ __forceinline__ float& gat(float* gs, int r, int c) { return gs[((r >> 1) * kGC + c) * 2 + (r & 1)]; }

// Clamp-to-edge for the Laplacian: the column and row just outside the
// image take the value of the nearest image pixel, so the stencil below
// needs no border cases (the Laplacian is only used at image pixels).
template <typename S>
__device__ __forceinline__ void replicate_borders(float* gs, int W, int H, int tx0, int ty0) {
  constexpr int kRows = S::ROWS;
  const int cl = 1 - tx0;          // gs column of x = -1 (valid when tx0 == 0)
  const int cr = W - tx0 + kHalo;  // gs column of x = W
  const int rt = 1 - ty0, rb = H - ty0 + kHalo;
  const bool left = tx0 == 0, right = cr < kGC, top = ty0 == 0, bottom = rb < kRows;
  if (!(left || right || top || bottom)) return;  // uniform over the CTA
  if (left || right) {
    for (int r = threadIdx.x; r < kRows; r += S::THREADS) {
      if (left) gat(gs, r, cl) = gat(gs, r, cl + 1);
      if (right) gat(gs, r, cr) = gat(gs, r, cr - 1);
    }
    __syncthreads();
  }
  if (top || bottom) {
    for (int c = threadIdx.x; c < kGC; c += S::THREADS) {
      if (top) gat(gs, rt, c) = gat(gs, rt + 1, c);
      if (bottom) gat(gs, rb, c) = gat(gs, rb - 1, c);
    }
    __syncthreads();
  }
}

// L_{o,k} = s_k^2 * (left + right + up + down - 4 centre) on row pairs; each
// thread walks one column down kRP / kLG row pairs with a sliding window.
// (The first and last tile rows of the band get a clamped, unused value.)
template <typename S>
__device__ __forceinline__ void laplacian(const float* gs, float s2k, float* L) {
  constexpr int kRP = S::RP, kLG = S::LG;
  constexpr int kPer = kRP / kLG;
  const float2 s2 = f2(s2k, s2k), m4 = f2(-4.0f, -4.0f);
  const float2* g = reinterpret_cast<const float2*>(gs);
  float2* out = reinterpret_cast<float2*>(L);
  for (int item = threadIdx.x; item < kLC * kLG; item += S::THREADS) {
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
template <typename S, typename StoreT>
__device__ __forceinline__ void store_level(const float* gs, StoreT* dst, int lpitch, int W, int H, int tx0,
                                            int ty0) {
  constexpr int kQ = kTX / 2;
  for (int i = threadIdx.x; i < (S::TY / 2) * kQ; i += S::THREADS) {
    const int m = i / kQ;            // tile rows 2m, 2m+1 = gs row pair m + 1
    const int c = (i - m * kQ) * 2;  // tile columns c, c+1 = gs columns c+2, c+3
    const int x = tx0 + c, y = ty0 + 2 * m;
    if (x >= W || y >= H) continue;
    const float4 v = *reinterpret_cast<const float4*>(gs + ((m + 1) * kGC + c + kHalo) * 2);
    store2(dst + (size_t)y * lpitch + x, v.x, v.z);
    if (y + 1 < H) store2(dst + (size_t)(y + 1) * lpitch + x, v.y, v.w);
  }
}

// Alg. 1: G_{o+1,0}[i][j] = G_{o,K-1}[2i][2j] for the even pixels of this
// tile, written transposed (to [j][i]) when the next octave is stored in the
// other orientation.  Consecutive threads write consecutive elements of a
// stored row either way (16 of a transposed row: 64 bytes).
template <typename S, typename StoreT>
__device__ __forceinline__ void store_decimated(const float* gs, StoreT* dst, int lpitch1, int W, int H,
                                                int tx0, int ty0, int dtr) {
  constexpr int kHX = kTX / 2, kHY = S::TY / 2;
  for (int i = threadIdx.x; i < kHX * kHY; i += S::THREADS) {
    const int r = dtr ? i % kHY : i / kHX;
    const int c = dtr ? i / kHY : i % kHX;
    const int y = ty0 + 2 * r, x = tx0 + 2 * c;
    if (y >= H || x >= W) continue;
    // tile row 2r is the first row of gs pair r + 1
    const float v = gs[((r + 1) * kGC + 2 * c + kHalo) * 2];
    store1(dst + (dtr ? (size_t)(x >> 1) * lpitch1 + (y >> 1) : (size_t)(y >> 1) * lpitch1 + (x >> 1)), v);
  }
}

// ------------------------------------------------ extremum in scale and space
struct Found {
  float xo, yo, so, resp, pss, ratio;
  int type;
};

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The admissible one of a pixel's two stationary points t0, t1 (values v,
// second derivatives s): inside [t_lo, t_hi], p'' != 0 and |p| >= T; when both
// are, the larger |p| wins, ties going to the smaller t.
__device__ __forceinline__ void pick_root(const DetectArgs& a, bool live, float t0, float t1, float v0, float v1,
                                          float s0, float s1, int& bt, float& tb) {
  const bool ok0 = live && t0 >= a.t_lo && t0 <= a.t_hi && s0 != 0.0f && fabsf(v0) >= a.T;
  const bool ok1 = live && t1 >= a.t_lo && t1 <= a.t_hi && s1 != 0.0f && fabsf(v1) >= a.T;
  const bool take1 = ok1 && (!ok0 || fabsf(v1) > fabsf(v0) || (fabsf(v1) == fabsf(v0) && t1 < t0));
  const float s = take1 ? s1 : s0;
  bt = (ok0 || ok1) ? (s < 0.0f ? 1 : -1) : 0;
  tb = (ok0 || ok1) ? (take1 ? t1 : t0) : 0.0f;
}

// S4 on a pair of pixels (phase 1): for each pixel, the admissible extremum
// of the cubic p(t) = a0 + a1 t + a2 t^2 + a3 t^3 with |p| >= T.  The roots of
// p'(t) = A t^2 + B t + C (A = 3 a3, B = 2 a2, C = a1) come from the
// cancellation-free form q = -(B + sign(B) sqrt(D)) / 2, t = q / A and C / q;
// they exist when D = B^2 - 4AC > 0.  With A = 0 the same formulas give q = -B
// and t = C / q = -C / B, the root of the linear derivative, while q / A is
// infinite and never admissible.  No branches: every pixel pair takes the same
// instruction stream, so the caller's unrolled pairs interleave.
// bt = +1 maximum, -1 minimum, 0 none.
__device__ __forceinline__ void cubic_extremum2(const DetectArgs& a, const float2 (&al)[4], bool live0,
                                                bool live1, int (&bt)[2], float (&tb)[2]) {
  const float2 A = mul2(f2(3.0f, 3.0f), al[3]), Bq = mul2(f2(2.0f, 2.0f), al[2]), C = al[1];
  const float2 D = fma2(mul2(f2(-4.0f, -4.0f), A), C, mul2(Bq, Bq));
  const float2 sq = f2(sqrt_approx(fmaxf(D.x, 0.0f)), sqrt_approx(fmaxf(D.y, 0.0f)));
  const float2 q = mul2(f2(-0.5f, -0.5f), add2(Bq, f2(copysignf(sq.x, Bq.x), copysignf(sq.y, Bq.y))));
  const float2 r0 = mul2(q, f2(rcp_approx(A.x), rcp_approx(A.y)));
  const float2 r1 = mul2(C, f2(rcp_approx(q.x), rcp_approx(q.y)));
  const float2 six_a3 = mul2(f2(6.0f, 6.0f), al[3]);
  // p'' and p at both roots, both pixels
  const float2 pdd0 = fma2(six_a3, r0, Bq), pdd1 = fma2(six_a3, r1, Bq);
  const float2 v0 = fma2(fma2(fma2(al[3], r0, al[2]), r0, al[1]), r0, al[0]);
  const float2 v1 = fma2(fma2(fma2(al[3], r1, al[2]), r1, al[1]), r1, al[0]);
  pick_root(a, live0 && D.x > 0.0f, r0.x, r1.x, v0.x, v1.x, pdd0.x, pdd1.x, bt[0], tb[0]);
  pick_root(a, live1 && D.y > 0.0f, r0.y, r1.y, v0.y, v1.y, pdd0.y, pdd1.y, bt[1], tb[1]);
}

// 8-neighbour test at the centre's t* and refinement (Alg. 1 stage B) for
// a pixel that passed phase 1 (phase 2).
template <typename S>
__device__ __forceinline__ bool refine_pixel(const DetectArgs& a, const float* Ls, int ly, int lx, int bt,
                                             float btv, int x, int y, Found& f) {
  constexpr int kRP = S::RP;
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

// Phase-1 survivors of a tile: packed (ly, lx, type) and t*.
struct Pending {
  int code;  // ly << 16 | lx << 1 | (type > 0)
  float t;
};

// Tile j of a CTA is described by info[j % 3]: while tile j is processed,
// info[(j + 1) % 3] drives the copy of its successor and the last warp fills
// info[(j + 2) % 3] during phase 2, so no thread waits on the plan's global
// loads.
struct TileShared {
  int n_pending;
  TileInfo info[3];
};

// Whether a variant copies FP32 input straight into its FP32 tile: the
// 128 x 16 variants do (their shared memory then fits two CTAs per SM).
template <typename S, typename InT>
constexpr bool kDirect = S::TY == 16 && std::is_same<InT, float>::value;

// Whether a variant runs a tile's detection (phases 1 and 2) during the
// next tile's first level passes: the 128 x 32 variants do.  The scale test
// and the refinement then share phases with the next tile's input staging
// and first y pass, so their latency-bound work overlaps the filters'
// multiply-adds, and a tile costs two block barriers fewer.  The tile's L
// levels stay in shared memory until the next tile's first Laplacian
// overwrites them; the survivors list has a region of its own (so the
// 184-column tiles of radii above 14, whose shared memory is full, do not).
template <typename S, int ic>
constexpr bool kDefer = S::TY == 32 && ic == 160;

// What the detection of a tile needs to know about it.
struct DetTile {
  int tx0, ty0, W, H, img, tr;
  unsigned bmask;
};

// ---- phase 1, per pixel pair (tile rows 2m, 2m+1 are L row pair m + 1):
// cubic coefficients of Eq. 3 on packed pairs, then the admissible extremum
// in scale; survivors are compacted into `pend` (count in *n_pending).
template <typename S, bool Masked>
__device__ __forceinline__ void detect_phase1(const DetectArgs& a, const float* Ls, const DetTile& t,
                                              Pending* pend, int* n_pending) {
  constexpr int kRP = S::RP, kThreads = S::THREADS;
  constexpr int kIt = (kTX * S::TY / 2) / kThreads;
  const int lane = threadIdx.x & 31;
  int bt[kIt][2];
  float tb[kIt][2];
  // all pixel pairs of the thread first (independent work in flight), then
  // the compaction
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int idx = it * kThreads + threadIdx.x;
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
    const int x = t.tx0 + lx, y0 = t.ty0 + 2 * m;
    // rows 2m, 2m + 1 lie in block row m / 8; a proposal may rule the block out
    const bool inx =
        x >= 1 && x < t.W - 1 && (!Masked || ((t.bmask >> ((m >> 3) * (kTX / 16) + (lx >> 4))) & 1u));
    cubic_extremum2(a, al2, inx && y0 >= 1 && y0 < t.H - 1, inx && y0 + 1 < t.H - 1, bt[it], tb[it]);
  }
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int idx = it * kThreads + threadIdx.x;
    const int m = idx / kTX, lx = idx - (idx / kTX) * kTX;
    const unsigned m0 = __ballot_sync(0xffffffffu, bt[it][0] != 0);
    const unsigned m1 = __ballot_sync(0xffffffffu, bt[it][1] != 0);
    if (m0 | m1) {
      int base = 0;
      if (lane == 0) base = atomicAdd(n_pending, __popc(m0) + __popc(m1));
      base = __shfl_sync(0xffffffffu, base, 0);
      const unsigned below = (1u << lane) - 1u;
      if (bt[it][0] != 0) {
        Pending e;
        e.code = ((2 * m) << 16) | (lx << 1) | (bt[it][0] > 0 ? 1 : 0);
        e.t = tb[it][0];
        pend[base + __popc(m0 & below)] = e;
      }
      if (bt[it][1] != 0) {
        Pending e;
        e.code = ((2 * m + 1) << 16) | (lx << 1) | (bt[it][1] > 0 ? 1 : 0);
        e.t = tb[it][1];
        pend[base + __popc(m0) + __popc(m1 & below)] = e;
      }
    }
  }
}

// ---- phase 2: neighbour test and refinement of the np survivors, densely;
// one queue reservation per warp and round.  The queue order does not
// matter: the selection orders candidates by a total order of its own.
template <typename S>
__device__ __forceinline__ void detect_phase2(const DetectArgs& a, const float* Ls, const DetTile& t,
                                              const Pending* pend, int np) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = warp * 32; i0 < np; i0 += S::THREADS) {
    const int i = i0 + lane;
    Found f;
    bool found = false;
    if (i < np) {
      const Pending e = pend[i];
      const int ly = e.code >> 16, lx = (e.code >> 1) & 0x7fff;
      found = refine_pixel<S>(a, Ls, ly, lx, (e.code & 1) ? 1 : -1, e.t, t.tx0 + lx, t.ty0 + ly, f);
    }
    const unsigned msk = __ballot_sync(0xffffffffu, found);
    if (msk == 0) continue;
    int base = 0;
    if (lane == 0) base = atomicAdd(a.cand_count + t.img, __popc(msk));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (found) {
      const int pos = base + __popc(msk & ((1u << lane) - 1u));
      if (pos < a.cand_cap) {
        Cand c;
        const bool tr = t.tr;  // image frame
        c.xo = tr ? f.yo : f.xo;
        c.yo = tr ? f.xo : f.yo;
        c.so = f.so;
        c.resp = f.resp;
        c.pss = f.pss;
        c.ratio = f.ratio;
        c.octave = (short)a.octave;
        c.type = (short)f.type;
        c.spare = 0;
        a.cands[(size_t)t.img * a.cand_cap + pos] = c;
      } else {
        atomicOr(a.status, kStatusCandOverflow);
      }
    }
  }
}

// Shared memory of the survivors list when it has a region of its own.
template <typename S, int ic>
constexpr size_t kPendBytes = kDefer<S, ic> ? sizeof(Pending) * kTX * S::TY : 0;

// Masked: the first octave under a block proposal (per-tile modes and block
// masks; 128 x 32 tiles only); the plain detector compiles without any of it.
template <typename S, typename InT, typename StoreT, int ic, bool Masked>
__global__ void __launch_bounds__(S::THREADS, S::MINB)
    detect_kernel(const __grid_constant__ DetectArgs a, int rm, int n_tiles) {
  static_assert(!Masked || S::TY == kTY, "block proposals are laid out on 128 x 32 tiles");
  constexpr bool Direct = kDirect<S, InT>;
  constexpr bool Defer = kDefer<S, ic>;
  constexpr int kRows = S::ROWS, kRP = S::RP, kWarps = S::WARPS, kThreads = S::THREADS;
  extern __shared__ float4 smem4[];
  __shared__ TileShared sh;
  const int IR = kRows + 2 * rm;
  const size_t raw_floats = Direct ? 0 : ((size_t)IR * ic * sizeof(InT) + 15) / 16 * 4;
  InT* raw = reinterpret_cast<InT*>(smem4);
  float* in = reinterpret_cast<float*>(smem4) + raw_floats;
  float* tmp = in + (size_t)IR * ic;
  float* gs = tmp + kRows * ic;
  float* Ls = gs + kRows * kGC;
  float* pend_region = Ls + kScales * kRows * kLC;
  int* prefix = reinterpret_cast<int*>(pend_region + kPendBytes<S, ic> / sizeof(float));
  // the survivors list: its own region (deferred detection), or `in` -- for
  // the direct variants, whose `in` is receiving the next tile, `tmp` and `gs`
  Pending* pend = reinterpret_cast<Pending*>(Defer ? pend_region : (Direct ? tmp : in));
  // where the next tile's rows land: the staging buffer, or (FP32 input of
  // the direct variants) the FP32 tile itself
  InT* land = Direct ? reinterpret_cast<InT*>(in) : raw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (int i = threadIdx.x; i <= a.n_images; i += kThreads) prefix[i] = a.tile_prefix[i] - a.tile_base;
  if (threadIdx.x == 0) sh.n_pending = 0;
  __syncthreads();

  int b = blockIdx.x;
  if (b >= n_tiles) return;
  if (threadIdx.x == 0) {
    tile_info<S, InT>(a, prefix, b, n_tiles, ic, &sh.info[0]);
    tile_info<S, InT>(a, prefix, b + gridDim.x, n_tiles, ic, &sh.info[1]);
  }
  __syncthreads();
  if (sh.info[0].bulk) issue_tile_copy<S, InT>(sh.info[0], ic, rm, land);

  DetTile prev;        // the tile whose detection is deferred to this one
  bool prev_det = false;
  prev.tx0 = prev.ty0 = prev.W = prev.H = prev.img = prev.tr = 0;
  prev.bmask = 0u;

  for (int slot = 0; b < n_tiles; b += gridDim.x, slot = slot == 2 ? 0 : slot + 1) {
    const TileInfo& cur = sh.info[slot];
    const TileInfo& nxt = sh.info[slot == 2 ? 0 : slot + 1];
    TileInfo* after = &sh.info[slot == 0 ? 2 : slot - 1];
    // ---- this tile's input into `in`, and (deferred) the scale test of
    // the previous tile
    if (cur.bulk) {  // uniform
      cp_async_wait_all();
      __syncthreads();
      if constexpr (Direct) replicate_in_place<S>(cur, ic, rm, in);
      else convert_raw<S, InT>(raw, cur, ic, rm, in);
    } else {
      load_tile_direct<S, InT>(cur, ic, rm, in);
    }
    if constexpr (Defer) {
      if (prev_det) detect_phase1<S, Masked>(a, Ls, prev, pend, &sh.n_pending);
    } else {
      if (threadIdx.x == 0) sh.n_pending = 0;
    }
    __syncthreads();
    // ---- next tile's input on its way while this one is processed (raw is
    // free: every thread is past convert_raw); the direct variants wait for
    // the last y pass to be done with `in`
    if constexpr (!Direct)
      if (nxt.bulk) issue_tile_copy<S, InT>(nxt, ic, rm, raw);

    const int W = cur.W, H = cur.H, lpitch = cur.lpitch, tx0 = cur.tx0, ty0 = cur.ty0;
    const long long dec_off = cur.dec_off;
    const int dec_pitch = cur.dec_pitch;
    StoreT* lev = reinterpret_cast<StoreT*>(a.levels) + cur.level_off;
    const size_t lstride = (size_t)lpitch * H;

    // what a block proposal leaves to do on this tile (uniform over the CTA):
    // everything, the levels only, or level 3 and the next octave's base
    const int mode = Masked ? a.tile_mode[a.tile_base + b] : kModeDetect;
    const unsigned bmask = Masked ? a.block_mask[a.tile_base + b] : 0xFFFFu;
    const int k0 = Masked && mode == kModeLevel3 ? kScales - 1 : 0;

    // ---- levels: the y pass of level k+1 shares a phase with the stores and
    // the Laplacian of level k; (deferred) the previous tile's refinement
    // shares the first y pass's phase -- its L levels are overwritten only by
    // this tile's first Laplacian
    vpass_dispatch<S, ic>(a.radius[k0], a.taps[k0], in, rm, tmp);
    if constexpr (Defer)
      if (prev_det) detect_phase2<S>(a, Ls, prev, pend, sh.n_pending);
    __syncthreads();
    if constexpr (Defer)
      if (threadIdx.x == 0) sh.n_pending = 0;  // read by the refinement above, rewritten by the next scale test
    if constexpr (Direct)
      if (k0 == kScales - 1 && nxt.bulk) issue_tile_copy<S, InT>(nxt, ic, rm, land);
    hpass_dispatch<S, ic>(a.radius[k0], a.taps[k0], tmp, gs);
    __syncthreads();
    for (int k = k0; k < kScales; ++k) {
      replicate_borders<S>(gs, W, H, tx0, ty0);
      if (k > 0 || a.write_level0) store_level<S, StoreT>(gs, lev + k * lstride, lpitch, W, H, tx0, ty0);
      if (k == kScales - 1 && dec_off >= 0)
        store_decimated<S, StoreT>(gs, reinterpret_cast<StoreT*>(a.levels) + dec_off, dec_pitch, W, H, tx0, ty0,
                                   cur.dec_tr);
      if (!Masked || mode == kModeDetect) laplacian<S>(gs, a.s2[k], Ls + (size_t)k * kRP * kLC * 2);
      if (k + 1 < kScales) vpass_dispatch<S, ic>(a.radius[k + 1], a.taps[k + 1], in, rm, tmp);
      // the tile after next is looked up by one lane while the others filter
      if (k == k0 && warp == kWarps - 1 && lane == 0)
        tile_info<S, InT>(a, prefix, b + 2 * gridDim.x, n_tiles, ic, after);
      __syncthreads();
      if (k + 1 < kScales) {
        // after the last y pass `in` is free: the direct variants start the
        // next tile's copies into it now
        if constexpr (Direct)
          if (k + 1 == kScales - 1 && nxt.bulk) issue_tile_copy<S, InT>(nxt, ic, rm, land);
        hpass_dispatch<S, ic>(a.radius[k + 1], a.taps[k + 1], tmp, gs);
        __syncthreads();
      }
    }

    DetTile t;
    t.tx0 = tx0;
    t.ty0 = ty0;
    t.W = W;
    t.H = H;
    t.img = cur.img;
    t.tr = cur.tr;
    t.bmask = bmask;
    const bool det = !Masked || mode == kModeDetect;
    if constexpr (Defer) {
      // the scale test and refinement of this tile run with the next one
      prev = t;
      prev_det = det;
    } else {
      if (det) {
        detect_phase1<S, Masked>(a, Ls, t, pend, &sh.n_pending);
        __syncthreads();
        detect_phase2<S>(a, Ls, t, pend, sh.n_pending);
      }
      // the pending list lives in `in` (or `tmp`), rewritten by the next tile
      __syncthreads();
    }
  }
  if constexpr (Defer) {
    // the last tile's detection
    if (prev_det) {
      detect_phase1<S, Masked>(a, Ls, prev, pend, &sh.n_pending);
      __syncthreads();
      detect_phase2<S>(a, Ls, prev, pend, sh.n_pending);
    }
  }
  cp_async_wait_all();  // nothing may still be landing in shared memory at exit
}

}  // namespace

// The input tile pitch: 128 + 2 Cm columns for radii up to 14 and up to 24.
static int tile_pitch(int max_radius) { return max_radius <= 14 ? 160 : 184; }

template <typename S>
static size_t detect_smem(int max_radius, int in_size, int n_images) {
  const int ic = tile_pitch(max_radius);
  const size_t pend = ic == 160 ? kPendBytes<S, 160> : kPendBytes<S, 184>;
  const size_t rows = (size_t)(S::ROWS + 2 * max_radius);
  const bool direct = S::TY == 16 && in_size == 4;
  const size_t raw = direct ? 0 : (rows * ic * in_size + 15) / 16 * 16;
  return raw + sizeof(float) * (rows * ic + (size_t)S::ROWS * ic + (size_t)S::ROWS * kGC +
                                (size_t)kScales * S::ROWS * kLC) +
         pend + sizeof(int) * (size_t)(n_images + 1);
}

// The launch of one variant: shared memory attribute, and a grid of
// persistent CTAs, as many per SM as fit (at most the tile count).
template <typename S, typename IN, typename ST, int IC, bool M>
static cudaError_t launch_variant(const DetectArgs& a, int n_tiles, int max_radius, int n_sms, cudaStream_t s) {
  const size_t smem = detect_smem<S>(max_radius, sizeof(IN), a.n_images);
  auto kern = detect_kernel<S, IN, ST, IC, M>;
  static LaunchCache cache;
  int per_sm = 0;
  cudaError_t e = prepare_launch(kern, cache, (int)smem, S::THREADS, &per_sm);
  if (e != cudaSuccess || n_tiles <= 0) return e;  // no tiles: only the kernel's set-up
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = n_tiles < n_sms * per_sm ? n_tiles : n_sms * per_sm;
  kern<<<grid, S::THREADS, smem, s>>>(a, max_radius, n_tiles);
  return cudaGetLastError();
}

// One variant for the input / storage types of an octave and the tile pitch
// of its radii (radii above 14, from a larger sigma0 than the default, only
// in variant A).
template <typename S, bool M>
static cudaError_t launch_typed(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms,
                                cudaStream_t s) {
  constexpr bool kWide = std::is_same<S, ShapeA>::value;
  const bool wide = tile_pitch(max_radius) != 160;
  if constexpr (kWide) {
    if (wide) {
      if (storage == CDVS_STORAGE_FP16) {
        if (a.octave == 0) return launch_variant<S, uint8_t, __half, 184, M>(a, n_tiles, max_radius, n_sms, s);
        if constexpr (M) return cudaErrorInvalidValue;
        else return launch_variant<S, __half, __half, 184, M>(a, n_tiles, max_radius, n_sms, s);
      }
      if (a.octave == 0) return launch_variant<S, uint8_t, float, 184, M>(a, n_tiles, max_radius, n_sms, s);
      if constexpr (M) return cudaErrorInvalidValue;
      else return launch_variant<S, float, float, 184, M>(a, n_tiles, max_radius, n_sms, s);
    }
  } else {
    if (wide) return cudaErrorInvalidValue;
  }
  if (storage == CDVS_STORAGE_FP16) {
    if (a.octave == 0) return launch_variant<S, uint8_t, __half, 160, M>(a, n_tiles, max_radius, n_sms, s);
    if constexpr (M) return cudaErrorInvalidValue;
    else return launch_variant<S, __half, __half, 160, M>(a, n_tiles, max_radius, n_sms, s);
  }
  if (a.octave == 0) return launch_variant<S, uint8_t, float, 160, M>(a, n_tiles, max_radius, n_sms, s);
  if constexpr (M) return cudaErrorInvalidValue;
  else return launch_variant<S, float, float, 160, M>(a, n_tiles, max_radius, n_sms, s);
}

}  // namespace cdvs
