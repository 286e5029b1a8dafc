// host_downstream.cpp -- the host (CPU) parts of the C ABI: the selection
// order of Eq. 5 and the descriptor transform + ternary quantisation of
// Sec. III-C.  Deterministic, FP64 arithmetic for the transform.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/cdvs.h"

namespace {

// Total order of the selection: |response| descending, then y, x, sigma,
// octave ascending (the relevance of Eq. 5 stands in as |p-hat|).
bool ranks_before(const cdvs_keypoint& a, const cdvs_keypoint& b) {
  const float ra = std::fabs(a.response), rb = std::fabs(b.response);
  if (ra != rb) return ra > rb;
  if (a.y != b.y) return a.y < b.y;
  if (a.x != b.x) return a.x < b.x;
  if (a.sigma != b.sigma) return a.sigma < b.sigma;
  return a.octave < b.octave;
}

// Order-8 transforms of one cell histogram (Sec. III-C): set A on cells with
// cx + cy even, set B on the others.
void transform_a(const double* h, double* v) {
  v[0] = (h[2] - h[6]) * 0.5;
  v[1] = (h[3] - h[7]) * 0.5;
  v[2] = (h[0] - h[1]) * 0.5;
  v[3] = (h[2] - h[3]) * 0.5;
  v[4] = (h[4] - h[5]) * 0.5;
  v[5] = (h[6] - h[7]) * 0.5;
  v[6] = ((h[0] + h[4]) - (h[2] + h[6])) * 0.25;
  v[7] = ((h[0] + h[2] + h[4] + h[6]) - (h[1] + h[3] + h[5] + h[7])) * 0.125;
}

void transform_b(const double* h, double* v) {
  v[0] = (h[0] - h[4]) * 0.5;
  v[1] = (h[1] - h[5]) * 0.5;
  v[2] = (h[7] - h[0]) * 0.5;
  v[3] = (h[1] - h[2]) * 0.5;
  v[4] = (h[3] - h[4]) * 0.5;
  v[5] = (h[5] - h[6]) * 0.5;
  v[6] = ((h[1] + h[5]) - (h[3] + h[7])) * 0.25;
  v[7] = ((h[0] + h[1] + h[2] + h[3]) - (h[4] + h[5] + h[6] + h[7])) * 0.125;
}

}  // namespace

extern "C" {

int32_t cdvs_rank_host(const cdvs_keypoint* pts, int32_t n, int32_t max_keypoints, int32_t* order) {
  if (!pts || !order || n <= 0 || max_keypoints <= 0) return 0;
  std::vector<int32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int32_t a, int32_t b) { return ranks_before(pts[a], pts[b]); });
  const int32_t m = std::min(n, max_keypoints);
  std::copy(idx.begin(), idx.begin() + m, order);
  return m;
}

cdvs_status cdvs_transform_ternary(const float* desc, int32_t n, const double* t_lo, const double* t_hi,
                                   int8_t* out, double* v_out) {
  if (n < 0 || (n > 0 && (!desc || !t_lo || !t_hi || !out))) return CDVS_INVALID_ARGUMENT;
  for (int32_t r = 0; r < n; ++r) {
    const float* d = desc + (size_t)r * 128;
    double v[128];
    for (int cy = 0; cy < 4; ++cy)
      for (int cx = 0; cx < 4; ++cx) {
        const int c = (cy * 4 + cx) * 8;
        double h[8];
        for (int j = 0; j < 8; ++j) h[j] = (double)d[c + j];
        if (((cx + cy) & 1) == 0) transform_a(h, v + c);
        else transform_b(h, v + c);
      }
    int8_t* q = out + (size_t)r * 128;
    for (int j = 0; j < 128; ++j) q[j] = (int8_t)(v[j] < t_lo[j] ? -1 : (v[j] > t_hi[j] ? 1 : 0));
    if (v_out)
      for (int j = 0; j < 128; ++j) v_out[(size_t)r * 128 + j] = v[j];
  }
  return CDVS_OK;
}

}  // extern "C"
