// dedupe_select.cu -- K3 + K10: per image, the cross-octave duplicate check
// of Alg. 1 stage C and the top-N selection of Eq. 5, in one CTA.
//
//   1. Candidates are bucketed into square cells at least as wide as the
//      largest duplicate window (one pixel of the coarsest octave), so every
//      duplicate of a candidate lies in its own or one of the 8 surrounding
//      cells (a counting sort through shared-memory cell counters).
//   2. A candidate is removed when an adjacent-octave candidate within
//      |dx|, |dy| <= 2^max(o_a, o_b) image px and |log2(sigma_a/sigma_b)| <=
//      dlog2 has a larger |response| (or an equal one from a finer octave).
//      All decisions use the original set, so the result does not depend on
//      the order in which candidates were queued.
//   3. The N-th largest |response| among the kept candidates is found by a
//      4-pass radix select on the IEEE bits; the candidates at or above it are
//      gathered and bitonic-sorted by (|response| desc, y, x, sigma, octave),
//      a total order, and the first N are written in rank order.  When more
//      candidates tie at the N-th |response| than the sort list holds, the
//      radix select continues over y, x, sigma and octave to find the N-th
//      entry of the total order itself, and only the entries up to it are
//      gathered: the result never depends on the queue order.
#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kSelThreads = 512;

// A tie-list entry, as two arrays: the keys (|response|, y, x, sigma in image
// px) in a float4 and (octave, candidate index) in an int2.
__device__ __forceinline__ bool ranks_before(const float4& ka, int oa, const float4& kb, int ob) {
  if (ka.x != kb.x) return ka.x > kb.x;
  if (ka.y != kb.y) return ka.y < kb.y;
  if (ka.z != kb.z) return ka.z < kb.z;
  if (ka.w != kb.w) return ka.w < kb.w;
  return oa < ob;
}

// exclusive scan of cnt[0..n) in place (block-wide); returns the total
__device__ int block_exclusive_scan(int* cnt, int n, int* warp_sums) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + kSelThreads - 1) / kSelThreads;
  const int b0 = min(tid * per, n), b1 = min(b0 + per, n);
  int local = 0;
  for (int i = b0; i < b1; ++i) local += cnt[i];
  int incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kSelThreads / 32 ? warp_sums[lane] : 0;
    int wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += v;
    }
    if (lane < kSelThreads / 32) warp_sums[lane] = wi - w;  // exclusive warp offsets
    if (lane == kSelThreads / 32 - 1) warp_sums[32] = wi;   // total
  }
  __syncthreads();
  int run = warp_sums[warp] + incl - local;
  for (int i = b0; i < b1; ++i) {
    const int c = cnt[i];
    cnt[i] = run;
    run += c;
  }
  const int total = warp_sums[32];
  __syncthreads();
  return total;
}

// Order-preserving 32-bit key of a float (ascending), -0 taken as +0.
__device__ __forceinline__ unsigned float_key(float f) {
  const unsigned b = __float_as_uint(f + 0.0f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// The `remaining`-th largest 32-bit key among the members (member(i, key)
// returns whether candidate i takes part and sets its key): four passes of 8
// bits over a shared 256-bucket histogram.  On return `remaining` is how many
// members with exactly the returned key are still needed (block-uniform).
template <typename Member>
__device__ unsigned radix_select_desc(int n, int& remaining, int* s_hist, int* s_misc, Member member) {
  const int tid = threadIdx.x;
  unsigned prefix = 0u, mask = 0u;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += kSelThreads) s_hist[i] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += kSelThreads) {
      unsigned key;
      if (!member(i, key)) continue;
      if ((key & mask) == prefix) atomicAdd(s_hist + ((key >> shift) & 255u), 1);
    }
    __syncthreads();
    // the digit d where the count of keys with digits d and above first
    // reaches `remaining`, scanning down from 255: lane l of warp 0 sums
    // digits 255 - 8l .. 248 - 8l, a warp scan gives the counts above each
    // lane's group, and the lane whose group crosses walks its 8 digits
    if (tid < 32) {
      const int lane = tid;
      int c[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        c[q] = s_hist[255 - 8 * lane - q];
        sum += c[q];
      }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int excl = incl - sum;
      if (lane == 31 && incl < remaining) {  // fewer keys than remaining: as a full scan would end
        s_misc[1] = 0;
        s_misc[2] = remaining - incl;
      }
      if (excl < remaining && remaining <= incl) {
        int cum = excl;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (cum + c[q] >= remaining) {
            s_misc[1] = 255 - 8 * lane - q;
            s_misc[2] = remaining - cum;
            break;
          }
          cum += c[q];
        }
      }
    }
    __syncthreads();
    prefix |= (unsigned)s_misc[1] << shift;
    mask |= 255u << shift;
    remaining = s_misc[2];
    __syncthreads();
  }
  return prefix;
}

__global__ void __launch_bounds__(kSelThreads) select_kernel(const __grid_constant__ SelectArgs a) {
  extern __shared__ float4 smem4[];
  __shared__ int warp_sums[33];
  __shared__ int s_hist[256];
  __shared__ int s_misc[4];
  const int img = blockIdx.x;
  const int tid = threadIdx.x;
  const ImgPlan* P = a.plans + img;
  const int W = P->W, H = P->H, n_oct = P->n_oct;
  const int n = min(a.cand_count[img], a.cand_cap);
  const Cand* C = a.cands + (size_t)img * a.cand_cap;
  int* order = a.order + (size_t)img * a.cand_cap;
  unsigned char* keep = a.keep + (size_t)img * a.cand_cap;
  float4* skey = a.skey + (size_t)img * a.cand_cap;
  unsigned char* soct = a.soct + (size_t)img * a.cand_cap;

  // ---- 1. cells of side cs (image px), cs >= 2^(n_oct-1)
  int cs = 1 << max(n_oct - 1, 0);
  while (((W + cs - 1) / cs) * ((H + cs - 1) / cs) > kMaxCells) cs <<= 1;
  const int gx = (W + cs - 1) / cs, gy = (H + cs - 1) / cs, ncell = gx * gy;
  const float inv_cs = 1.0f / (float)cs;
  int* cell = reinterpret_cast<int*>(smem4);  // ncell + 1 counters -> ends
  for (int i = tid; i <= ncell; i += kSelThreads) cell[i] = 0;
  __syncthreads();
  // a candidate of an octave the image does not have takes no part (the
  // callers' records are checked here, not trusted)
  auto valid = [&](int i) { return C[i].octave >= 0 && C[i].octave < n_oct; };
  bool bad_input = false;
  for (int i = tid; i < n; i += kSelThreads) {
    if (!valid(i)) {
      bad_input = true;
      continue;
    }
    const float s = (float)(1 << C[i].octave);
    const int cx = min(max((int)floorf(C[i].xo * s * inv_cs), 0), gx - 1);
    const int cy = min(max((int)floorf(C[i].yo * s * inv_cs), 0), gy - 1);
    atomicAdd(cell + cy * gx + cx, 1);
  }
  if (bad_input) atomicOr(a.status, kStatusBadInput);
  __syncthreads();
  block_exclusive_scan(cell, ncell, warp_sums);
  for (int i = tid; i < n; i += kSelThreads) {
    if (!valid(i)) continue;
    const float s = (float)(1 << C[i].octave);
    const int cx = min(max((int)floorf(C[i].xo * s * inv_cs), 0), gx - 1);
    const int cy = min(max((int)floorf(C[i].yo * s * inv_cs), 0), gy - 1);
    const int pos = atomicAdd(cell + cy * gx + cx, 1);  // after this, cell[c] = end of cell c
    order[pos] = i;
    // the compact copy the check reads, in cell order (the same products as
    // the check would form from the record)
    skey[pos] = make_float4(C[i].xo * s, C[i].yo * s, C[i].so * s, fabsf(C[i].resp));
    soct[pos] = (unsigned char)C[i].octave;
  }
  __syncthreads();

  // ---- 2. cross-octave duplicates, walked in cell order: neighbouring lanes
  // take neighbouring candidates, so they read the same runs of the sorted
  // copy (cached lines), and no read depends on another
  for (int i = tid; i < n; i += kSelThreads)
    if (!valid(i)) keep[i] = 0;
  const int nv = cell[ncell - 1];  // candidates that took part in the sort
  int kept_local = 0;
  for (int p = tid; p < nv; p += kSelThreads) {
    const float4 ka = skey[p];
    const int oa = soct[p];
    const float xa = ka.x, ya = ka.y, siga = ka.z, ra = ka.w;
    const int cx = min(max((int)floorf(xa * inv_cs), 0), gx - 1);
    const int cy = min(max((int)floorf(ya * inv_cs), 0), gy - 1);
    bool k = true;
    for (int yy = max(cy - 1, 0); yy <= min(cy + 1, gy - 1) && k; ++yy)
      for (int xx = max(cx - 1, 0); xx <= min(cx + 1, gx - 1) && k; ++xx) {
        const int c = yy * gx + xx;
        const int beg = c == 0 ? 0 : cell[c - 1], end = cell[c];
        for (int j = beg; j < end; ++j) {
          const int ob = soct[j];
          const int d = oa - ob;
          if (d != 1 && d != -1) continue;
          const float4 kb = skey[j];
          const float win = (float)(1 << max(oa, ob));
          if (!(fabsf(xa - kb.x) <= win && fabsf(ya - kb.y) <= win)) continue;
          if (!(fabsf(log2f(siga / kb.z)) <= a.dlog2)) continue;
          const float rb = kb.w;
          if (rb > ra || (rb == ra && ob < oa)) {
            k = false;
            break;
          }
        }
      }
    keep[order[p]] = k ? 1 : 0;
    kept_local += k ? 1 : 0;
  }
  if (tid == 0) s_misc[0] = 0;
  __syncthreads();
  atomicAdd(s_misc, kept_local);
  __syncthreads();
  const int M = s_misc[0];
  const int N = a.N;

  // ---- 3. radix select of the N-th largest |response| (IEEE bits of a
  // non-negative float order like the floats themselves)
  unsigned thr = 0u;
  if (M > N) {
    int remaining = N;
    thr = radix_select_desc(n, remaining, s_hist, s_misc, [&](int i, unsigned& key) {
      key = __float_as_uint(fabsf(C[i].resp));
      return keep[i] != 0;
    });
  }

  // ---- gather candidates at or above the threshold and sort them
  float4* key = smem4;  // reuses the cell counters
  int2* aux = reinterpret_cast<int2*>(key + a.list_cap);
  // tie keys (y, x, sigma, octave) of a candidate, image px; the total order
  // takes them ascending, so they are selected complemented (largest first)
  auto tie_key = [&](int i, int k) -> unsigned {
    const float s = (float)(1 << C[i].octave);
    if (k == 0) return ~float_key(C[i].yo * s);
    if (k == 1) return ~float_key(C[i].xo * s);
    if (k == 2) return ~float_key(C[i].so * s);
    return ~(unsigned)(C[i].octave + 0x8000);
  };
  unsigned tkey[4] = {0u, 0u, 0u, 0u};
  int n_tie_keys = 0;  // 0: every candidate at thr is gathered
  int L = 0;
  for (int pass = 0; pass < 2; ++pass) {
    if (tid == 0) s_misc[3] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += kSelThreads) {
      if (!keep[i]) continue;
      const float ar = fabsf(C[i].resp);
      const unsigned ab = __float_as_uint(ar);
      if (ab < thr) continue;
      if (ab == thr && n_tie_keys > 0) {
        // at the threshold: only the ties up to the N-th entry of the total order
        bool in = true;
        for (int k = 0; k < 4; ++k) {
          const unsigned t = tie_key(i, k);
          if (t != tkey[k]) {
            in = t > tkey[k];
            break;
          }
        }
        if (!in) continue;
      }
      const int pos = atomicAdd(s_misc + 3, 1);
      if (pos >= a.list_cap) continue;
      const float s = (float)(1 << C[i].octave);
      key[pos] = make_float4(ar, C[i].yo * s, C[i].xo * s, C[i].so * s);
      aux[pos] = make_int2(C[i].octave, i);
    }
    __syncthreads();
    const int gathered = s_misc[3];
    __syncthreads();
    if (gathered <= a.list_cap || pass == 1) {
      if (tid == 0 && gathered > a.list_cap) atomicOr(a.status, kStatusSelectOverflow);
      L = min(gathered, a.list_cap);
      break;
    }
    // More candidates tie at the N-th |response| than the list holds: find
    // the N-th entry of the total order among the ties (radix select on y,
    // x, sigma, octave in turn), so the list gets exactly the N first ones
    // whatever the order the candidates were queued in.
    int above = 0;
    for (int i = tid; i < n; i += kSelThreads)
      above += keep[i] && __float_as_uint(fabsf(C[i].resp)) > thr;
    __syncthreads();
    if (tid == 0) s_misc[0] = 0;
    __syncthreads();
    atomicAdd(s_misc, above);
    __syncthreads();
    int remaining = N - s_misc[0];
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
      const int kk = k;
      tkey[k] = radix_select_desc(n, remaining, s_hist, s_misc, [&](int i, unsigned& t) {
        if (!keep[i] || __float_as_uint(fabsf(C[i].resp)) != thr) return false;
        for (int j = 0; j < kk; ++j)
          if (tie_key(i, j) != tkey[j]) return false;
        t = tie_key(i, kk);
        return true;
      });
    }
    n_tie_keys = 4;
  }
  int Pn = 1;
  while (Pn < L) Pn <<= 1;
  for (int i = L + tid; i < Pn; i += kSelThreads) {  // padding that ranks last
    key[i] = make_float4(-1.0f, 0.0f, 0.0f, 0.0f);
    aux[i] = make_int2(0x7fffffff, -1);
  }
  __syncthreads();
  // bitonic sort of the entries in place
  for (int k = 2; k <= Pn; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < Pn; i += kSelThreads) {
        const int l = i ^ j;
        if (l > i) {
          const float4 ki = key[i], kl = key[l];
          const int2 ai = aux[i], al = aux[l];
          const bool asc = (i & k) == 0;  // ascending in "rank" order
          const bool swap = asc ? ranks_before(kl, al.x, ki, ai.x) : ranks_before(ki, ai.x, kl, al.x);
          if (swap) {
            key[i] = kl;
            key[l] = ki;
            aux[i] = al;
            aux[l] = ai;
          }
        }
      }
      __syncthreads();
    }
  }
  const int cnt = min(N, L);
  Cand* out = a.sel + (size_t)img * N;
  for (int r = tid; r < cnt; r += kSelThreads) out[r] = C[aux[r].y];
  if (tid == 0) a.sel_count[img] = cnt;
}

}  // namespace

// The tie list holds the N selected candidates and any that tie with the
// N-th: 2N entries (at least 1024, at most kSelectList) of 24 bytes, sorted
// in place.  Sized by N, the shared memory of N = 300 is the 32 KB of cell
// counters, and three CTAs share an SM (as many as the registers allow), so a
// 256-image batch selects in one wave; N = 2000 takes 96 KB, two CTAs per SM.
// A fixed 4096-entry list with a separate permutation (115 KB) had allowed
// one CTA per SM.
cudaError_t launch_select(const SelectArgs& args, int n_images, cudaStream_t s) {
  if (n_images <= 0) return cudaSuccess;
  SelectArgs a = args;
  a.list_cap = 1024;
  while (a.list_cap < 2 * a.N && a.list_cap < kSelectList) a.list_cap <<= 1;
  const size_t smem_cells = sizeof(int) * (kMaxCells + 1);
  const size_t smem_list = (sizeof(float4) + sizeof(int2)) * (size_t)a.list_cap;
  const size_t smem = smem_cells > smem_list ? smem_cells : smem_list;
  static LaunchCache cache;
  cudaError_t e = prepare_launch(select_kernel, cache, (int)smem, kSelThreads, nullptr);
  if (e != cudaSuccess) return e;
  select_kernel<<<n_images, kSelThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cdvs
