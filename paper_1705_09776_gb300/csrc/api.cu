// api.cu -- the C ABI of include/cdvs.h: context, parameter checks, batch
// planning (octave sizes, level arena layout, tile lists), workspace, host <->
// device staging, and the launch sequence
//   K1 detect (one launch per octave, all images)
//   K3+K10 cross-octave check + selection (one CTA per image)
//   K5 orientation, packing scan, K6 descriptors
// Every step of the method runs in the kernels; this file only moves bytes.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cdvs_internal.cuh"

using namespace cdvs;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct HostBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// What one call stages: page-locked copies of the small per-call tables (one
// buffer per upload site, so no upload overwrites another one still in
// flight), the device copy of host images, and the device copy of records
// bound for host memory.  Calls alternate between two sets.  The host tables
// of a set are rewritten only after the call two back that used it has
// finished (`done`), its input copy only after that call's detection
// (`in_free`), its output copy only after that call's records reached the
// host (`out_free`); so an asynchronous call stages and enqueues its batch
// while the previous one is still running.
struct StageSet {
  HostBuf plans, prefix, prop, jobs, plans2;
  HostBuf small;  // status word + record total
  DevBuf input, out_kp, out_desc, out_count;
  cudaEvent_t done = nullptr, in_free = nullptr, out_free = nullptr, packed = nullptr;
};

// An asynchronous call with host outputs whose records still have to be
// copied out (the copies are enqueued once its record total is known).
struct PendingReadback {
  bool on = false;
  int set = 0, n = 0;
  cdvs_keypoint* kp = nullptr;
  float* desc = nullptr;
  int32_t* count = nullptr;
};

struct ProfRec {
  int stage, launches;
  cudaEvent_t a, b;
};

}  // namespace

constexpr int kMaxInputChunks = 4;

struct Upload {
  void* dst;
  const void* src;
  size_t bytes;
};

struct cdvs_ctx {
  int device = 0;
  int n_sms = 0;
  std::string err;
  DevBuf levels, cands, cand_count, order, keep, skey, soct, sel, sel_count, ori_theta, ori_count, rec_off,
      rec_total, plans, tile_prefix, status, input, dump, stage_kp, stage_desc;
  // learned block proposal: parameters, per-call image table, logits, tile modes, training workspace
  DevBuf prop_theta, prop_imgs, prop_logits, prop_mode, prop_ws;
  DevBuf resized, resize_jobs;  // S0: resized images and their job table
  DevBuf scfv_model, scfv_desc, scfv_q, scfv_out, scfv_off;  // SCFV model and scratch (scfv_q: the gradient operands)
  DevBuf out_counters;  // per output group: slot claims, scan CTAs done, first record (+1)
  bool scfv_set = false;
  // the per-call staging sets (StageSet) and the CUDA graph that
  // device-resident extractions are replayed through
  StageSet hset[2];
  int cur_set = 0;
  bool async_open = false;  // CDVS_ASYNC extractions since the last cdvs_wait
  PendingReadback pend;
  cudaStream_t d2h_stream = nullptr;  // record copies of asynchronous calls
  StageSet& hs() { return hset[cur_set]; }
  bool graph = false;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t gstream = nullptr;  // capture stream when the caller passes the legacy default stream
  cudaEvent_t gev = nullptr;
  bool prop_set = false;
  std::vector<ImgPlan> h_plans;
  std::vector<int> h_prefix;
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  // host inputs go up in image chunks on copy_stream, each chunk's octave-0
  // detection waiting for its chunk only
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ready[kMaxInputChunks + 1] = {};
  int n_chunks = 1;                        // of the current call
  int chunk_begin[kMaxInputChunks + 1] = {};
  std::vector<Upload> uploads[kMaxInputChunks];  // empty: inputs already on the device
  // candidate queue capacity per image: at least this many (grown after a
  // call whose queue overflowed), and the capacity of the last call
  // K1 work-shape tuner: per class of octave launches (first octave or the
  // later ones, storage type, level radii) the measured time per tile of
  // each variant; the variant of every octave of the current call
  struct TuneClass {
    int later, storage;
    int radii[kScales];
    float ms_per_tile[kDetectVariants];  // < 0: not measured yet
    int inflight[kDetectVariants];       // measurements enqueued, not read back
  };
  struct Measure {
    int cls, variant;
    long long tiles;
    cudaEvent_t a, b;
  };
  std::vector<TuneClass> tune;
  std::vector<Measure> measures;
  int variant_mode = -1;  // cdvs_set_detect_variant: -1 tuned, else fixed
  int oct_variant[kMaxOctaves] = {};
  int cap_floor = 0;
  int cap_fixed = 0;  // cdvs_set_candidate_capacity; 0: from the image size
  int last_cap = 0;
  bool overflow_rerun = false;  // inside the re-run of an overflowed call
};

namespace {

enum Mode { kExtract, kCandidates, kDescribe, kScaleSpace };

cdvs_status fail(cdvs_ctx* c, cdvs_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

cdvs_status cuda_fail(cdvs_ctx* c, cudaError_t e, const char* what) {
  if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? CDVS_OUT_OF_MEMORY : CDVS_CUDA_ERROR;
}

cudaEvent_t take_event(cdvs_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Stage timing: an event before the stage's launches and one after them, on
// the stream the kernels run on.
cudaEvent_t prof_begin(cdvs_ctx* c, cudaStream_t s) {
  if (!c->prof) return nullptr;
  cudaEvent_t e = take_event(c);
  if (e) cudaEventRecord(e, s);
  return e;
}

void prof_end(cdvs_ctx* c, int stage, int launches, cudaEvent_t a, cudaStream_t s) {
  if (!c->prof || !a) return;
  cudaEvent_t b = take_event(c);
  if (!b) return;
  cudaEventRecord(b, s);
  c->recs.push_back(ProfRec{stage, launches, a, b});
}

// Fault injection for tests of the error paths (cdvs_inject_alloc_failures):
// the next g_fail_allocs workspace allocations fail as cudaMalloc would when
// the device is out of memory.
std::atomic<int> g_fail_allocs{0};
// the next g_skip_products cdvs_scfv calls leave their tensor-core products
// unissued, so the posterior kernel's bounded wait runs out (a testing hook)
std::atomic<int> g_skip_products{0};

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (bytes <= b.bytes) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  const size_t nb = bytes + bytes / 4;
  for (int f = g_fail_allocs.load(); f > 0;)
    if (g_fail_allocs.compare_exchange_weak(f, f - 1)) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(&b.p, nb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  b.bytes = nb;
  return cudaSuccess;
}

cudaError_t ensure_host(HostBuf& b, size_t bytes);

// Host table -> device through a page-locked copy (capturable in a graph).
cudaError_t upload(HostBuf& stage, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = ensure_host(stage, bytes);
  if (e != cudaSuccess) return e;
  std::memcpy(stage.p, src, bytes);
  return cudaMemcpyAsync(dst, stage.p, bytes, cudaMemcpyHostToDevice, s);
}

cudaError_t ensure_host(HostBuf& b, size_t bytes) {
  if (bytes <= b.bytes) return cudaSuccess;
  if (b.p) cudaFreeHost(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMallocHost(&b.p, bytes);
  if (e != cudaSuccess) return e;
  b.bytes = bytes;
  return cudaSuccess;
}

// ---- method constants computed on the host (double), passed to the kernels

double scale_k(const cdvs_params& p, int k) {
  return (double)p.sigma0 * std::pow(2.0, (double)k / (double)(p.scales_per_octave - 1));
}

// Blur added to the octave base to reach s_k: the input carries sigma_in,
// a decimated base carries sigma0 (in its own pixels).
double tau_of(const cdvs_params& p, int octave, int k) {
  const double s = scale_k(p, k);
  const double b = octave == 0 ? (double)p.sigma_in : (double)p.sigma0;
  const double v = s * s - b * b;
  return v > 0.0 ? std::sqrt(v) : 0.0;
}

// One side (index 0..r) of the sampled Gaussian on [-r, r], r = ceil(4 tau),
// normalised to unit sum.
int gauss_taps(double tau, float* one_side) {
  if (tau <= 0.0) {
    one_side[0] = 1.0f;
    return 0;
  }
  const int r = (int)std::ceil(4.0 * tau);
  if (r > kMaxRadius) return -1;
  double w[kMaxRadius + 1], sum = 0.0;
  for (int j = 0; j <= r; ++j) {
    w[j] = std::exp(-(double)(j * j) / (2.0 * tau * tau));
    sum += j == 0 ? w[j] : 2.0 * w[j];
  }
  for (int j = 0; j <= r; ++j) one_side[j] = (float)(w[j] / sum);
  return r;
}

// Cubic through the K = 4 samples (s_k, L_k) in the centred variable
// t = sigma - tc: a = Vc^-1 L with Vc[k][i] = (s_k - tc)^i (Eq. 2-3 with the
// interpolating beta; centring only improves FP32 conditioning).
bool centred_fit(const cdvs_params& p, float B[4][kScales], float& tc, float& tlo, float& thi) {
  const int K = kScales;
  double s[kScales];
  for (int k = 0; k < K; ++k) s[k] = scale_k(p, k);
  const double c = 0.5 * (s[0] + s[K - 1]);
  double A[4][8];
  for (int k = 0; k < K; ++k) {
    double v = 1.0;
    for (int i = 0; i < 4; ++i) {
      A[k][i] = v;
      v *= s[k] - c;
    }
    for (int j = 0; j < 4; ++j) A[k][4 + j] = k == j ? 1.0 : 0.0;
  }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int i = col + 1; i < 4; ++i)
      if (std::fabs(A[i][col]) > std::fabs(A[piv][col])) piv = i;
    if (A[piv][col] == 0.0) return false;
    for (int j = 0; j < 8; ++j) std::swap(A[col][j], A[piv][j]);
    const double d = A[col][col];
    for (int j = 0; j < 8; ++j) A[col][j] /= d;
    for (int i = 0; i < 4; ++i) {
      if (i == col) continue;
      const double f = A[i][col];
      for (int j = 0; j < 8; ++j) A[i][j] -= f * A[col][j];
    }
  }
  // A[:, 4:] = Vc^-1: a_i = sum_k Vc^-1[i][k] L_k
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < K; ++k) B[i][k] = (float)A[i][4 + k];
  tc = (float)c;
  tlo = (float)(s[0] - c);
  thi = (float)(s[K - 1] - c);
  return true;
}

cdvs_status check_params(cdvs_ctx* c, const cdvs_params* p) {
  if (!p) return fail(c, CDVS_INVALID_ARGUMENT, "params is NULL");
  if (p->scales_per_octave != kScales) return fail(c, CDVS_INVALID_ARGUMENT, "scales_per_octave must be 4");
  if (p->num_octaves < 1 || p->num_octaves > kMaxOctaves)
    return fail(c, CDVS_INVALID_ARGUMENT, "num_octaves must be in 1..12");
  if (!(p->sigma0 > 0.0f) || !(p->sigma_in >= 0.0f) || !(p->sigma_in <= p->sigma0))
    return fail(c, CDVS_INVALID_ARGUMENT, "need 0 <= sigma_in <= sigma0, sigma0 > 0");
  if (!(p->contrast_T >= 0.0f) || !(p->edge_r > 0.0f) || !(p->offset_max > 0.0f))
    return fail(c, CDVS_INVALID_ARGUMENT, "contrast_T >= 0, edge_r > 0, offset_max > 0 required");
  if (!(p->ori_radius > 0.0f) || !(p->ori_weight_sigma > 0.0f) || !(p->desc_radius > 0.0f) ||
      !(p->cell_side > 0.0f) || !(p->desc_weight_sigma > 0.0f) || !(p->ori_peak_ratio >= 0.0f) ||
      !(p->dedupe_dlog2 >= 0.0f))
    return fail(c, CDVS_INVALID_ARGUMENT, "description radii, weights and ratios must be positive");
  if (p->max_keypoints < 1 || p->max_keypoints > kMaxSelect)
    return fail(c, CDVS_INVALID_ARGUMENT, "max_keypoints must be in 1..2048");
  if (p->max_orientations < 1 || p->max_orientations > kMaxOri)
    return fail(c, CDVS_INVALID_ARGUMENT, "max_orientations must be in 1..8");
  if (p->storage != CDVS_STORAGE_FP32 && p->storage != CDVS_STORAGE_FP16)
    return fail(c, CDVS_INVALID_ARGUMENT, "storage must be CDVS_STORAGE_FP32 or CDVS_STORAGE_FP16");
  if (p->use_proposal != 0 && p->use_proposal != 1) return fail(c, CDVS_INVALID_ARGUMENT, "use_proposal must be 0 or 1");
  if (p->max_side != 0 && (p->max_side < 16 || p->max_side > 32768))
    return fail(c, CDVS_INVALID_ARGUMENT, "max_side must be 0 or 16..32768");
  if (p->use_proposal && !(p->proposal_threshold > 0.0f && p->proposal_threshold < 1.0f))
    return fail(c, CDVS_INVALID_ARGUMENT, "proposal_threshold must be in (0, 1)");
  float t[kMaxRadius + 1];
  for (int o = 0; o < 2; ++o)
    for (int k = 0; k < kScales; ++k)
      if (gauss_taps(tau_of(*p, o, k), t) < 0)
        return fail(c, CDVS_INVALID_ARGUMENT, "a level filter radius exceeds 24 (sigma0 too large)");
  return CDVS_OK;
}

size_t elem_size(int storage) { return storage == CDVS_STORAGE_FP16 ? 2 : 4; }

// Octave sizes, level arena layout and tile lists of a batch.
cdvs_status plan_batch(cdvs_ctx* c, int n, const cdvs_image_desc* sizes, const cdvs_params& p,
                       long long& level_elems, int& max_oct, long long& max_pixels) {
  c->h_plans.assign(n, ImgPlan{});
  level_elems = 0;
  max_oct = 0;
  max_pixels = 0;
  for (int i = 0; i < n; ++i) {
    const cdvs_image_desc& d = sizes[i];
    if (d.width < 16 || d.height < 16 || d.width > 32768 || d.height > 32768)
      return fail(c, CDVS_UNSUPPORTED_SIZE, "image " + std::to_string(i) + ": sides must be in 16..32768");
    if (d.pitch_bytes < d.width) return fail(c, CDVS_INVALID_ARGUMENT, "pitch_bytes < width");
    ImgPlan& P = c->h_plans[i];
    P.W = d.width;
    P.H = d.height;
    P.pitch = d.pitch_bytes;
    int w = d.width, h = d.height, no = 0;
    for (int o = 0; o < p.num_octaves; ++o) {
      if (w < 3 || h < 3) break;
      OctPlan& op = P.oct[o];
      // past the first octave (whose input is the caller's image), store the
      // octave transposed when that takes fewer 128 x 32 tiles
      auto tiles = [](int tw, int th) { return ((tw + kTX - 1) / kTX) * ((th + kTY - 1) / kTY); };
      op.tr = o > 0 && tiles(h, w) < tiles(w, h);
      op.W = op.tr ? h : w;
      op.H = op.tr ? w : h;
      op.lpitch = (op.W + 7) & ~7;
      op.tiles_x = (op.W + kTX - 1) / kTX;
      op.tiles_y = (op.H + kTY - 1) / kTY;
      op.level_off = level_elems;
      level_elems += ((long long)kScales * op.lpitch * op.H + 63) & ~63LL;
      ++no;
      w = (w + 1) / 2;
      h = (h + 1) / 2;
    }
    P.n_oct = no;
    max_oct = std::max(max_oct, no);
    max_pixels = std::max(max_pixels, (long long)d.width * d.height);
  }
  return CDVS_OK;
}

// Tiles of octave o of image i with the tile rows of a K1 variant (tiles are
// 128 wide in every variant).
long long variant_tiles(const ImgPlan& P, int o, int variant) {
  if (o >= P.n_oct) return 0;
  const int ty = detect_variant_rows(variant);
  return (long long)P.oct[o].tiles_x * ((P.oct[o].H + ty - 1) / ty);
}

// Per octave, the first tile of every image in the launch's tile order, for
// the variant that runs the octave (c->oct_variant).
void build_prefix(cdvs_ctx* c, int n, int max_oct) {
  c->h_prefix.assign((size_t)kMaxOctaves * (n + 1), 0);
  for (int o = 0; o < max_oct; ++o) {
    int* pre = c->h_prefix.data() + (size_t)o * (n + 1);
    pre[0] = 0;
    for (int i = 0; i < n; ++i) pre[i + 1] = pre[i] + (int)variant_tiles(c->h_plans[i], o, c->oct_variant[o]);
  }
}

// ---- the K1 work-shape tuner
//
// Every variant computes the same levels and candidates bit for bit, so the
// tuner measures them on the caller's own calls: while a class of octave
// launches has an unmeasured variant, each call runs one such variant and
// times its launches with CUDA events on the call's stream (read back by a
// later call, without synchronising); once every variant has a time per
// tile, each octave takes the variant whose time per tile times its tile
// count for the batch is smallest.  The first octave is measured only on
// calls whose images are already on the device (its launches wait for
// uploads otherwise).

int tune_class(cdvs_ctx* c, bool later, int storage, const int* radii) {
  for (size_t i = 0; i < c->tune.size(); ++i) {
    const auto& t = c->tune[i];
    if (t.later == (int)later && t.storage == storage && std::equal(radii, radii + kScales, t.radii)) return (int)i;
  }
  cdvs_ctx::TuneClass t;
  t.later = later;
  t.storage = storage;
  std::copy(radii, radii + kScales, t.radii);
  for (int v = 0; v < kDetectVariants; ++v) {
    t.ms_per_tile[v] = -1.0f;
    t.inflight[v] = 0;
  }
  c->tune.push_back(t);
  return (int)c->tune.size() - 1;
}

// Measurements whose launches have finished become times per tile (the
// smallest seen per variant).
void harvest_measures(cdvs_ctx* c) {
  std::vector<cdvs_ctx::Measure> keep;
  for (auto& m : c->measures) {
    const cudaError_t q = cudaEventQuery(m.b);
    if (q == cudaErrorNotReady) {
      keep.push_back(m);
      continue;
    }
    float ms = 0.0f;
    auto& t = c->tune[m.cls];
    --t.inflight[m.variant];
    if (q == cudaSuccess && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess && m.tiles > 0) {
      const float per = ms / (float)m.tiles;
      float& cur = t.ms_per_tile[m.variant];
      cur = cur < 0.0f ? per : std::min(cur, per);
    }
    cudaGetLastError();
    c->pool.push_back(m.a);
    c->pool.push_back(m.b);
  }
  c->measures.swap(keep);
}

bool class_tuned(const cdvs_ctx::TuneClass& t) {
  for (int v = 0; v < kDetectVariants; ++v)
    if (t.ms_per_tile[v] < 0.0f) return false;
  return true;
}

// The variant of every octave of this call; the classes this call measures
// (cls, variant) in `measure` (at most one per class).
void choose_variants(cdvs_ctx* c, int n, int max_oct, const cdvs_params& p, bool masked0, bool device_inputs,
                     std::vector<std::pair<int, int>>& measure) {
  measure.clear();
  harvest_measures(c);
  for (int o = 0; o < max_oct; ++o) {
    int radii[kScales];
    float taps[kMaxRadius + 1];
    for (int k = 0; k < kScales; ++k) radii[k] = gauss_taps(tau_of(p, o, k), taps);
    // radii above 14 (a sigma0 above the default's) and the first octave
    // under a block proposal run on variant 0 only
    const bool only0 = (o == 0 && masked0) || *std::max_element(radii, radii + kScales) > 14;
    if (c->variant_mode >= 0 || only0) {
      c->oct_variant[o] = only0 ? 0 : c->variant_mode;
      continue;
    }
    const size_t n_classes = c->tune.size();
    const int cls = tune_class(c, o > 0, p.storage, radii);
    auto& t = c->tune[cls];
    if (c->tune.size() > n_classes) {
      // a new class: load every variant's kernel now, so no timed launch
      // pays for loading it
      DetectArgs a;
      std::memset(&a, 0, sizeof(a));
      a.octave = o;
      a.n_images = n;
      const int maxr = *std::max_element(radii, radii + kScales);
      for (int u = 0; u < kDetectVariants; ++u) launch_detect(a, 0, maxr, p.storage, c->n_sms, u, nullptr);
      cudaGetLastError();
    }
    int v = -1;
    for (const auto& m : measure)
      if (m.first == cls) v = m.second;  // a later octave of a class measured by this call
    if (v < 0 && !class_tuned(t) && (o > 0 || device_inputs)) {
      for (int u = 0; u < kDetectVariants && v < 0; ++u)
        if (t.ms_per_tile[u] < 0.0f && t.inflight[u] == 0) v = u;
      if (v >= 0) measure.push_back({cls, v});
    }
    if (v < 0) {
      // the measured variant with the least predicted time for this batch
      double best = 0.0;
      v = 0;
      for (int u = 0; u < kDetectVariants; ++u) {
        if (t.ms_per_tile[u] < 0.0f) continue;
        long long tiles = 0;
        for (int i = 0; i < n; ++i) tiles += variant_tiles(c->h_plans[i], o, u);
        const double cost = (double)tiles * t.ms_per_tile[u];
        if (best == 0.0 || cost < best) {
          best = cost;
          v = u;
        }
      }
    }
    c->oct_variant[o] = v;
  }
}

int cand_capacity(long long max_pixels, int fixed, int floor) {
  long long cap = fixed > 0 ? fixed : std::max(4096LL, (max_pixels / 16 + 1023) & ~1023LL);
  if (floor > cap) cap = ((long long)floor + 1023) & ~1023LL;
  return (int)std::min(cap, 1LL << 22);
}

// After a call whose candidate queue overflowed: the queue counters kept
// counting past the capacity, so the largest count is the capacity that
// holds every candidate.
void grow_cap_floor(cdvs_ctx* c, const int* counts, int n) {
  int mx = 0;
  for (int i = 0; i < n; ++i) mx = std::max(mx, counts[i]);
  c->cap_floor = std::max(c->cap_floor, mx);
}

// Uploads images (if on the host) and the plans; returns the plan of image i
// pointing at device memory.
// Host images are uploaded in up to kMaxInputChunks chunks of whole images on
// the context's copy stream; each chunk's copies are issued just before the
// first octave's detection of that chunk (issue_upload), which waits for them,
// so the detection of chunk k overlaps the upload of chunk k + 1 -- also for
// pageable memory, whose copies hold the host thread while they are staged.
cdvs_status stage_inputs(cdvs_ctx* c, int n, const uint8_t* const* images, const cdvs_image_desc* sizes,
                         uint32_t flags, cudaStream_t s) {
  cudaError_t e;
  c->n_chunks = 1;
  c->chunk_begin[0] = 0;
  c->chunk_begin[1] = n;
  for (auto& u : c->uploads) u.clear();
  if (flags & CDVS_INPUT_DEVICE) {
    for (int i = 0; i < n; ++i) c->h_plans[i].src = images[i];
  } else {
    size_t total = 0;
    std::vector<size_t> off(n + 1);
    for (int i = 0; i < n; ++i) {
      off[i] = total;
      total += (size_t)sizes[i].pitch_bytes * sizes[i].height;
      total = (total + 255) & ~(size_t)255;
    }
    off[n] = total;
    DevBuf& input = c->hs().input;
    if ((e = ensure(input, total)) != cudaSuccess) return cuda_fail(c, e, "input staging");
    uint8_t* base = static_cast<uint8_t*>(input.p);
    if (!c->copy_stream) {
      if ((e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(c, e, "copy stream");
      for (cudaEvent_t& ev : c->ready)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
          return cuda_fail(c, e, "copy events");
    }
    // chunks only pay off for batches that fill the GPU several times over
    c->n_chunks = n >= 64 ? kMaxInputChunks : 1;
    for (int k = 0; k <= c->n_chunks; ++k) c->chunk_begin[k] = (int)((long long)n * k / c->n_chunks);
    for (int k = 0; k < c->n_chunks; ++k) {
      const int i0 = c->chunk_begin[k], i1 = c->chunk_begin[k + 1];
      // back-to-back host images of one size go up in one copy
      bool contiguous = i1 > i0;
      const size_t isz = i1 > i0 ? (size_t)sizes[i0].pitch_bytes * sizes[i0].height : 0;
      for (int i = i0 + 1; i < i1 && contiguous; ++i)
        contiguous = sizes[i].pitch_bytes == sizes[i0].pitch_bytes && sizes[i].height == sizes[i0].height &&
                     images[i] == images[i0] + (size_t)(i - i0) * isz && off[i] == off[i0] + (size_t)(i - i0) * isz;
      if (contiguous) {
        c->uploads[k].push_back(Upload{base + off[i0], images[i0], isz * (i1 - i0)});
      } else {
        for (int i = i0; i < i1; ++i)
          c->uploads[k].push_back(Upload{base + off[i], images[i], (size_t)sizes[i].pitch_bytes * sizes[i].height});
      }
    }
    // the copies start once the last detection that read this staging buffer
    // (two calls back) is done
    if ((e = cudaStreamWaitEvent(c->copy_stream, c->hs().in_free, 0)) != cudaSuccess)
      return cuda_fail(c, e, "copy ordering");
    for (int i = 0; i < n; ++i) c->h_plans[i].src = base + off[i];
  }
  if ((e = ensure(c->plans, sizeof(ImgPlan) * n)) != cudaSuccess) return cuda_fail(c, e, "plans");
  if ((e = ensure(c->tile_prefix, sizeof(int) * c->h_prefix.size())) != cudaSuccess)
    return cuda_fail(c, e, "tile lists");
  if ((e = upload(c->hs().plans, c->plans.p, c->h_plans.data(), sizeof(ImgPlan) * n, s)) != cudaSuccess)
    return cuda_fail(c, e, "plan upload");
  if ((e = upload(c->hs().prefix, c->tile_prefix.p, c->h_prefix.data(), sizeof(int) * c->h_prefix.size(), s)) !=
      cudaSuccess)
    return cuda_fail(c, e, "tile list upload");
  return CDVS_OK;
}

// Chunk k of the host images on its way, and s waiting for it.
cudaError_t issue_upload(cdvs_ctx* c, int k, cudaStream_t s) {
  if (c->uploads[k].empty()) return cudaSuccess;
  cudaError_t e;
  for (const Upload& u : c->uploads[k])
    if ((e = cudaMemcpyAsync(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, c->copy_stream)) != cudaSuccess)
      return e;
  if ((e = cudaEventRecord(c->ready[k], c->copy_stream)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(s, c->ready[k], 0);
}

cdvs_status run_detect(cdvs_ctx* c, int n, const cdvs_params& p, int max_oct, int cap, cudaStream_t s,
                       const std::vector<std::pair<int, int>>& measure, const uint8_t* tile_mode = nullptr,
                       const uint16_t* block_mask = nullptr) {
  cudaError_t e;
  DetectArgs a;
  std::memset(&a, 0, sizeof(a));
  a.plans = static_cast<const ImgPlan*>(c->plans.p);
  a.n_images = n;
  a.levels = c->levels.p;
  a.cands = static_cast<Cand*>(c->cands.p);
  a.cand_count = static_cast<int*>(c->cand_count.p);
  a.cand_cap = cap;
  a.status = static_cast<int*>(c->status.p);
  for (int k = 0; k < kScales; ++k) {
    const double sk = scale_k(p, k);
    a.s2[k] = (float)(sk * sk);
  }
  if (!centred_fit(p, a.B, a.tc, a.t_lo, a.t_hi)) return fail(c, CDVS_INVALID_ARGUMENT, "degenerate scales");
  a.T = p.contrast_T;
  a.edge_lim = (float)(((double)p.edge_r + 1.0) * ((double)p.edge_r + 1.0) / (double)p.edge_r);
  a.offset_max = p.offset_max;
  cudaEvent_t m_ev[2] = {nullptr, nullptr};
  int m_idx[2] = {-1, -1};
  for (int o = 0; o < max_oct; ++o) {
    a.octave = o;
    a.write_level0 = o == 0 ? 1 : 0;
    a.tile_mode = o == 0 ? tile_mode : nullptr;
    a.block_mask = o == 0 ? block_mask : nullptr;
    int maxr = 0;
    for (int k = 0; k < kScales; ++k) {
      float t1[kMaxRadius + 1];
      a.radius[k] = gauss_taps(tau_of(p, o, k), t1);
      for (int j = 0; j <= std::max(a.radius[k], 0); ++j) a.taps[k][j] = make_float2(t1[j], t1[j]);
      maxr = std::max(maxr, a.radius[k]);
    }
    const int* prefix = c->h_prefix.data() + (size_t)o * (n + 1);
    const int* d_prefix = static_cast<const int*>(c->tile_prefix.p) + (size_t)o * (n + 1);
    // octave 0 runs per input chunk, each launch after its chunk's upload
    const int parts = o == 0 ? c->n_chunks : 1;
    cudaEvent_t ev0 = o == 0 ? prof_begin(c, s) : nullptr;
    // a tuner measurement starts at the first octave of its group (octave 0
    // alone, or octaves 1 .. max_oct - 1, which share radii and input type)
    const int g = o > 0 ? 1 : 0;
    if (o <= 1)
      for (size_t j = 0; j < measure.size(); ++j)
        if (c->tune[measure[j].first].later == g && measure[j].second == c->oct_variant[o] &&
            (m_ev[g] = take_event(c)) != nullptr) {
          m_idx[g] = (int)j;
          cudaEventRecord(m_ev[g], s);
          break;
        }
    for (int k = 0; k < parts; ++k) {
      const int i0 = parts > 1 ? c->chunk_begin[k] : 0, i1 = parts > 1 ? c->chunk_begin[k + 1] : n;
      if (o == 0 && (e = issue_upload(c, k, s)) != cudaSuccess) return cuda_fail(c, e, "image upload");
      a.plans = static_cast<const ImgPlan*>(c->plans.p) + i0;
      a.cands = static_cast<Cand*>(c->cands.p) + (size_t)i0 * cap;
      a.cand_count = static_cast<int*>(c->cand_count.p) + i0;
      a.n_images = i1 - i0;
      a.tile_prefix = d_prefix + i0;
      a.tile_base = prefix[i0];
      const int n_tiles = prefix[i1] - prefix[i0];
      if (n_tiles > 0 && (e = launch_detect(a, n_tiles, maxr, p.storage, c->n_sms, c->oct_variant[o], s)) != cudaSuccess)
        return cuda_fail(c, e, "detect launch");
    }
    if (o == 0) prof_end(c, 5, parts, ev0, s);
    // ... and ends after its last octave
    if (m_ev[g] && o == (g ? max_oct - 1 : 0)) {
      cudaEvent_t mb = take_event(c);
      if (mb) {
        cudaEventRecord(mb, s);
        long long tiles = 0;
        for (int q = g; q <= o; ++q) tiles += c->h_prefix[(size_t)q * (n + 1) + n];
        const auto& m = measure[m_idx[g]];
        c->measures.push_back(cdvs_ctx::Measure{m.first, m.second, tiles, m_ev[g], mb});
        ++c->tune[m.first].inflight[m.second];
      } else {
        c->pool.push_back(m_ev[g]);
      }
      m_ev[g] = nullptr;
    }
  }
  return CDVS_OK;
}

DescribeArgs describe_args(cdvs_ctx* c, int n, const cdvs_params& p) {
  DescribeArgs d;
  std::memset(&d, 0, sizeof(d));
  d.plans = static_cast<const ImgPlan*>(c->plans.p);
  d.levels = c->levels.p;
  d.sel = static_cast<const Cand*>(c->sel.p);
  d.sel_count = static_cast<const int*>(c->sel_count.p);
  d.N = p.max_keypoints;
  d.n_images = n;
  d.ori_theta = static_cast<float*>(c->ori_theta.p);
  d.ori_count = static_cast<int*>(c->ori_count.p);
  d.rec_off = static_cast<int*>(c->rec_off.p);
  d.rec_total = static_cast<int*>(c->rec_total.p);
  d.status = static_cast<int*>(c->status.p);
  d.sigma0 = p.sigma0;
  d.upright = p.upright;
  d.max_ori = p.max_orientations;
  d.ori_radius = p.ori_radius;
  d.ori_ratio = p.ori_peak_ratio;
  d.ori_wsig = p.ori_weight_sigma;
  d.desc_radius = p.desc_radius;
  d.cell_side = p.cell_side;
  d.desc_wsig = p.desc_weight_sigma;
  // the largest sampling disc of a detected point (sigma <= 2 sigma0 in
  // octave px) plus the gradient margin; larger discs read global memory
  const double smax = 2.0 * (double)p.sigma0 * (1.0 + 1e-3);
  const double rmax = std::max((double)p.desc_radius, p.upright ? 0.0 : (double)p.ori_radius) * smax;
  d.patch_side = std::min(2 * (int)std::ceil(rmax) + 3, 55);
  d.stage_kp = static_cast<cdvs_keypoint*>(c->stage_kp.p);
  d.stage_desc = static_cast<float*>(c->stage_desc.p);
  return d;
}

cdvs_status map_status(cdvs_ctx* c, int st) {
  if (st & kStatusTimeout) {
    c->err = "a bounded device-side wait gave up (asynchronous copy did not complete)";
    return CDVS_DEVICE_TIMEOUT;
  }
  if (st & (kStatusCandOverflow | kStatusSelectOverflow | kStatusOutTruncated)) {
    std::string m;
    if (st & kStatusCandOverflow) m += "candidate queue full; ";
    if (st & kStatusSelectOverflow) m += "selection tie list full; ";
    if (st & kStatusOutTruncated) m += "output capacity reached; ";
    c->err = m;
    return CDVS_CAPACITY_TRUNCATED;
  }
  c->err.clear();
  return CDVS_OK;
}

struct PointsIn {
  const cdvs_keypoint* pts;
  const int32_t* counts;
  int32_t stride;
};

// The shared pipeline behind cdvs_extract / cdvs_candidates / cdvs_describe.
const uint32_t* prop_frag(cdvs_ctx* c) {
  const size_t pbytes = (sizeof(float) * kPropParams + 255) & ~(size_t)255;
  return reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(c->prop_theta.p) + pbytes);
}

// The proposal network's per-image table (sizes of every layer, first logit)
// for images whose device pixels are srcs[i]; returns the number of logits.
size_t prop_table(int n, const cdvs_image_desc* sizes, const uint8_t* const* srcs, std::vector<PropImage>& t,
                  int& max_th, int& max_tw) {
  t.resize(n);
  size_t off = 0;
  max_th = max_tw = 0;
  for (int i = 0; i < n; ++i) {
    PropImage& q = t[i];
    q.src = srcs[i];
    q.W = sizes[i].width;
    q.H = sizes[i].height;
    q.pitch = sizes[i].pitch_bytes;
    q.H1 = (q.H + 1) / 2;
    q.W1 = (q.W + 1) / 2;
    q.H2 = (q.H1 + 1) / 2;
    q.W2 = (q.W1 + 1) / 2;
    q.Th = (q.H + 15) / 16;
    q.Tw = (q.W + 15) / 16;
    q.logit_off = (int)off;
    off += (size_t)q.Th * q.Tw;
    max_th = std::max(max_th, q.Th);
    max_tw = std::max(max_tw, q.Tw);
  }
  return off;
}

// Block proposal for the batch already staged on the device (h_plans[i].src):
// logits, then the first octave's tile modes in c->prop_mode.
cdvs_status run_proposal_mask(cdvs_ctx* c, int n, const cdvs_image_desc* sizes, const cdvs_params& p,
                              cudaStream_t s) {
  if (!c->prop_set) return fail(c, CDVS_INVALID_ARGUMENT, "use_proposal set but no cdvs_set_proposal call");
  std::vector<const uint8_t*> srcs(n);
  for (int i = 0; i < n; ++i) srcs[i] = c->h_plans[i].src;
  std::vector<PropImage> t;
  int max_th, max_tw;
  const size_t n_logits = prop_table(n, sizes, srcs.data(), t, max_th, max_tw);
  const int n_tiles = c->h_prefix[n];
  int max_tiles = 0;
  for (int i = 0; i < n; ++i) max_tiles = std::max(max_tiles, c->h_plans[i].oct[0].tiles_x * c->h_plans[i].oct[0].tiles_y);
  cudaError_t e;
  if ((e = ensure(c->prop_imgs, sizeof(PropImage) * n)) != cudaSuccess ||
      (e = ensure(c->prop_logits, sizeof(float) * n_logits)) != cudaSuccess ||
      (e = ensure(c->prop_mode, (size_t)n_tiles * 4 + n_logits)) != cudaSuccess)
    return cuda_fail(c, e, "proposal workspace");
  if ((e = upload(c->hs().prop, c->prop_imgs.p, t.data(), sizeof(PropImage) * n, s)) != cudaSuccess)
    return cuda_fail(c, e, "proposal table upload");
  const PropImage* d_t = static_cast<const PropImage*>(c->prop_imgs.p);
  if ((e = launch_proposal_infer(d_t, n, max_th, max_tw, static_cast<const float*>(c->prop_theta.p), prop_frag(c),
                                 static_cast<float*>(c->prop_logits.p), s)) != cudaSuccess)
    return cuda_fail(c, e, "proposal launch");
  // a descriptor disc of a first-octave point reaches this far (image px)
  const double reach = std::max(p.desc_radius, p.ori_radius) * 2.0 * p.sigma0 * 1.001 + 2.0;
  const int ny = (int)std::ceil(reach / kTY), nx = (int)std::ceil(reach / kTX);
  const double thr = p.proposal_threshold;
  const float zt = (float)std::log(thr / (1.0 - thr));
  // prop_mode: modes (n_tiles) | spare (n_tiles) | block masks (2 n_tiles) ...
  // the spare bytes hold the per-tile detect flags, then near flags per block
  uint8_t* mb = static_cast<uint8_t*>(c->prop_mode.p);
  if ((e = launch_tile_mode(d_t, static_cast<const ImgPlan*>(c->plans.p), static_cast<const int*>(c->tile_prefix.p),
                            n, max_th * max_tw, max_tiles, static_cast<const float*>(c->prop_logits.p), zt, 1, ny,
                            nx, mb, reinterpret_cast<uint16_t*>(mb + 2 * (size_t)n_tiles), mb + 4 * (size_t)n_tiles,
                            mb + (size_t)n_tiles, s)) != cudaSuccess)
    return cuda_fail(c, e, "tile mode launch");
  return CDVS_OK;
}

// S0 target size: the larger side becomes max_side, the other side is scaled
// and rounded to the nearest integer, ties to even (at least 1).
void resize_target(int W, int H, int max_side, int& W2, int& H2) {
  W2 = W;
  H2 = H;
  if (max_side <= 0 || std::max(W, H) <= max_side) return;
  auto rhe = [](long long num, long long den) {
    long long q = num / den, r = num - q * den;
    if (2 * r > den || (2 * r == den && (q & 1))) ++q;
    return q;
  };
  if (W >= H) {
    W2 = max_side;
    H2 = (int)std::max(1LL, rhe((long long)H * max_side, W));
  } else {
    H2 = max_side;
    W2 = (int)std::max(1LL, rhe((long long)W * max_side, H));
  }
}

// S0 on the device: every resized image into c->resized (row pitch a
// multiple of 16), and the plans pointed at them.
cdvs_status run_resize(cdvs_ctx* c, int n, const cdvs_image_desc* sizes, const std::vector<cdvs_image_desc>& eff,
                       cudaStream_t s) {
  std::vector<ResizeJob> jobs;
  size_t total = 0;
  std::vector<size_t> off(n, 0);
  for (int i = 0; i < n; ++i)
    if (eff[i].width != sizes[i].width || eff[i].height != sizes[i].height) {
      off[i] = total;
      total += ((size_t)eff[i].pitch_bytes * eff[i].height + 255) & ~(size_t)255;
    }
  cudaError_t e;
  if ((e = ensure(c->resized, total)) != cudaSuccess) return cuda_fail(c, e, "resize buffer");
  int max_pixels = 0;
  for (int i = 0; i < n; ++i)
    if (eff[i].width != sizes[i].width || eff[i].height != sizes[i].height) {
      ResizeJob j;
      j.src = c->h_plans[i].src;
      j.W = sizes[i].width;
      j.H = sizes[i].height;
      j.pitch = sizes[i].pitch_bytes;
      j.dst = static_cast<uint8_t*>(c->resized.p) + off[i];
      j.W2 = eff[i].width;
      j.H2 = eff[i].height;
      j.pitch2 = eff[i].pitch_bytes;
      jobs.push_back(j);
      c->h_plans[i].src = j.dst;
      max_pixels = std::max(max_pixels, j.H2);  // rows
    }
  if (jobs.empty()) return CDVS_OK;
  if ((e = ensure(c->resize_jobs, sizeof(ResizeJob) * jobs.size())) != cudaSuccess ||
      (e = upload(c->hs().jobs, c->resize_jobs.p, jobs.data(), sizeof(ResizeJob) * jobs.size(), s)) != cudaSuccess ||
      (e = launch_resize(static_cast<const ResizeJob*>(c->resize_jobs.p), (int)jobs.size(), max_pixels, s)) !=
          cudaSuccess ||
      (e = upload(c->hs().plans2, c->plans.p, c->h_plans.data(), sizeof(ImgPlan) * n, s)) != cudaSuccess)
    return cuda_fail(c, e, "resize");
  return CDVS_OK;
}

// The pending readback of an asynchronous call with host outputs: waits
// until the call's records are packed (its record total is then in the set's
// page-locked word), copies them out on the readback stream, and marks the
// set's output copy free again after the copies.
cdvs_status flush_readback(cdvs_ctx* c) {
  PendingReadback& r = c->pend;
  if (!r.on) return CDVS_OK;
  r.on = false;
  StageSet& set = c->hset[r.set];
  cudaError_t e;
  if (!c->d2h_stream && (e = cudaStreamCreateWithFlags(&c->d2h_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(c, e, "readback stream");
  if ((e = cudaEventSynchronize(set.packed)) != cudaSuccess) return cuda_fail(c, e, "readback");
  const int total = static_cast<const int*>(set.small.p)[1];
  cudaStream_t q = c->d2h_stream;
  if ((e = cudaStreamWaitEvent(q, set.packed, 0)) != cudaSuccess ||
      (e = cudaMemcpyAsync(r.count, set.out_count.p, sizeof(int) * r.n, cudaMemcpyDeviceToHost, q)) != cudaSuccess ||
      (total > 0 && (e = cudaMemcpyAsync(r.kp, set.out_kp.p, sizeof(cdvs_keypoint) * (size_t)total,
                                         cudaMemcpyDeviceToHost, q)) != cudaSuccess) ||
      (total > 0 && (e = cudaMemcpyAsync(r.desc, set.out_desc.p, sizeof(float) * 128 * (size_t)total,
                                         cudaMemcpyDeviceToHost, q)) != cudaSuccess) ||
      (e = cudaEventRecord(set.out_free, q)) != cudaSuccess)
    return cuda_fail(c, e, "readback");
  return CDVS_OK;
}

cdvs_status run(cdvs_ctx* c, Mode mode, int n, const uint8_t* const* images, const cdvs_image_desc* sizes,
                const cdvs_params* params, const PointsIn* pin, cdvs_keypoint* kp_out, float* desc_out,
                int32_t capacity, int32_t* kp_count, uint32_t flags, cudaStream_t s) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  cdvs_status st = check_params(c, params);
  if (st != CDVS_OK) return st;
  const cdvs_params& p = *params;
  if (n < 0) return fail(c, CDVS_INVALID_ARGUMENT, "n_images < 0");
  if (n > kMaxBatch) return fail(c, CDVS_INVALID_ARGUMENT, "at most 4096 images per call");
  if (n == 0) {
    c->err.clear();
    return CDVS_OK;
  }
  if (!images || !sizes) return fail(c, CDVS_INVALID_ARGUMENT, "images or sizes is NULL");
  for (int i = 0; i < n; ++i)
    if (!images[i]) return fail(c, CDVS_INVALID_ARGUMENT, "image pointer is NULL");
  if (mode != kScaleSpace && (!kp_out || !kp_count || capacity < 0 || (mode != kCandidates && !desc_out)))
    return fail(c, CDVS_INVALID_ARGUMENT, "output pointer is NULL or capacity < 0");
  if (mode == kCandidates && (flags & CDVS_OUTPUT_DEVICE))
    return fail(c, CDVS_INVALID_ARGUMENT, "cdvs_candidates writes host memory only");
  const bool async = (flags & CDVS_ASYNC) != 0;
  if (async && mode != kExtract) return fail(c, CDVS_INVALID_ARGUMENT, "CDVS_ASYNC is for cdvs_extract only");
  if (!async && c->async_open)
    return fail(c, CDVS_INVALID_ARGUMENT, "asynchronous extractions are pending: call cdvs_wait first");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  // the host staging set of this call, free once the call two back is done;
  // the guard marks it in use up to this call's last enqueued work, on every
  // return path
  c->cur_set ^= 1;
  StageSet& hset = c->hs();
  if (hset.done && (e = cudaEventSynchronize(hset.done)) != cudaSuccess) return cuda_fail(c, e, "staging set");
  // records of this set still waiting to go out (an asynchronous call with
  // host outputs two calls back, followed by one with device outputs) leave
  // before this call's packing can overwrite them
  if (c->pend.on && c->pend.set == c->cur_set && (st = flush_readback(c)) != CDVS_OK) return st;
  for (cudaEvent_t* ev : {&hset.done, &hset.in_free, &hset.out_free, &hset.packed})
    if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(c, e, "staging set");
  struct SetGuard {
    cudaEvent_t ev;
    cudaStream_t& s;
    ~SetGuard() { cudaEventRecord(ev, s); }
  } set_guard{hset.done, s};

  // S0: the sizes the method sees
  std::vector<cdvs_image_desc> eff(sizes, sizes + n);
  bool any_resize = false;
  for (int i = 0; i < n; ++i) {
    int W2, H2;
    resize_target(sizes[i].width, sizes[i].height, p.max_side, W2, H2);
    if (W2 != sizes[i].width || H2 != sizes[i].height) {
      if (sizes[i].pitch_bytes < sizes[i].width) return fail(c, CDVS_INVALID_ARGUMENT, "pitch_bytes < width");
      eff[i].width = W2;
      eff[i].height = H2;
      eff[i].pitch_bytes = (W2 + 15) & ~15;
      any_resize = true;
    }
  }
  long long level_elems, max_pixels;
  int max_oct;
  if ((st = plan_batch(c, n, eff.data(), p, level_elems, max_oct, max_pixels)) != CDVS_OK) return st;
  const bool proposal = p.use_proposal && (mode == kExtract || mode == kCandidates);
  // K1's work shape per octave (measured by this call while a class is being
  // tuned), then the tile lists of that shape
  std::vector<std::pair<int, int>> measure;
  choose_variants(c, n, max_oct, p, proposal, (flags & CDVS_INPUT_DEVICE) || any_resize, measure);
  build_prefix(c, n, max_oct);
  const int cap = cand_capacity(max_pixels, c->cap_fixed, c->cap_floor);
  c->last_cap = cap;
  const int N = p.max_keypoints;
  const size_t slots = (size_t)n * N;
  if ((e = ensure(c->levels, (size_t)level_elems * elem_size(p.storage))) != cudaSuccess ||
      (e = ensure(c->cands, sizeof(Cand) * (size_t)n * cap)) != cudaSuccess ||
      (e = ensure(c->cand_count, sizeof(int) * n)) != cudaSuccess ||
      (e = ensure(c->order, sizeof(int) * (size_t)n * cap)) != cudaSuccess ||
      (e = ensure(c->keep, (size_t)n * cap)) != cudaSuccess ||
      (e = ensure(c->skey, sizeof(float4) * (size_t)n * cap)) != cudaSuccess ||
      (e = ensure(c->soct, (size_t)n * cap)) != cudaSuccess ||
      (e = ensure(c->sel, sizeof(Cand) * slots)) != cudaSuccess ||
      (e = ensure(c->sel_count, sizeof(int) * n)) != cudaSuccess ||
      (e = ensure(c->ori_theta, sizeof(float) * slots * kMaxOri)) != cudaSuccess ||
      (e = ensure(c->ori_count, sizeof(int) * slots)) != cudaSuccess ||
      (e = ensure(c->rec_off, sizeof(int) * (slots + 2 * (size_t)n + 1))) != cudaSuccess ||
      (e = ensure(c->rec_total, sizeof(int) * 4)) != cudaSuccess ||
      (e = ensure(c->status, sizeof(int) * 4)) != cudaSuccess ||
      (e = ensure(c->stage_kp, sizeof(cdvs_keypoint) * slots * p.max_orientations)) != cudaSuccess ||
      (e = ensure(c->stage_desc, sizeof(float) * 128 * slots * p.max_orientations)) != cudaSuccess ||
      (e = ensure_host(c->hs().small, sizeof(int) * (4 + kMaxOutGroups + 1))) != cudaSuccess)
    return cuda_fail(c, e, "workspace");

  // Device-resident extraction can run as one CUDA graph: the stream work
  // below is captured, the cached executable graph is updated in place (or
  // instantiated again when the work changed shape) and launched.
  // (calls that measure a K1 variant run their launches directly)
  const bool graph = c->graph && mode == kExtract && (flags & CDVS_INPUT_DEVICE) && (flags & CDVS_OUTPUT_DEVICE) &&
                     !c->prof && measure.empty();
  struct CaptureGuard {  // ends an abandoned capture on early returns
    cudaStream_t s;
    bool on = false;
    ~CaptureGuard() {
      if (!on) return;
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
  } capture{s};
  const cudaStream_t caller_s = s;
  if (graph) {
    if (!s) {  // the legacy default stream cannot be captured: work on our own stream after it
      if (!c->gstream && ((e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking)) != cudaSuccess ||
                          (e = cudaEventCreateWithFlags(&c->gev, cudaEventDisableTiming)) != cudaSuccess))
        return cuda_fail(c, e, "graph stream");
      if ((e = cudaEventRecord(c->gev, s)) != cudaSuccess || (e = cudaStreamWaitEvent(c->gstream, c->gev, 0)) != cudaSuccess)
        return cuda_fail(c, e, "graph stream");
      s = c->gstream;
      capture.s = s;
    }
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
      return cuda_fail(c, e, "graph capture");
    capture.on = true;
  }
  if ((st = stage_inputs(c, n, images, sizes, flags, s)) != CDVS_OK) return st;
  // the status bits of asynchronous calls accumulate until cdvs_wait
  if ((e = cudaMemsetAsync(c->cand_count.p, 0, sizeof(int) * n, s)) != cudaSuccess ||
      (!c->async_open && (e = cudaMemsetAsync(c->status.p, 0, sizeof(int) * 4, s)) != cudaSuccess))
    return cuda_fail(c, e, "memset");
  cudaEvent_t ev = prof_begin(c, s);
  const uint8_t* tile_mode = nullptr;
  const uint16_t* block_mask = nullptr;
  if (proposal || any_resize) {
    // the resize and the network read the whole batch: every upload first
    for (int k = 0; k < c->n_chunks; ++k)
      if ((e = issue_upload(c, k, s)) != cudaSuccess) return cuda_fail(c, e, "image upload");
    for (auto& u : c->uploads) u.clear();
    c->n_chunks = 1;
    c->chunk_begin[1] = n;
  }
  if (any_resize && (st = run_resize(c, n, sizes, eff, s)) != CDVS_OK) return st;
  if (proposal) {
    cudaEvent_t evp = prof_begin(c, s);
    if ((st = run_proposal_mask(c, n, eff.data(), p, s)) != CDVS_OK) return st;
    prof_end(c, 6, 2, evp, s);
    tile_mode = static_cast<const uint8_t*>(c->prop_mode.p);
    block_mask = reinterpret_cast<const uint16_t*>(tile_mode + 2 * (size_t)c->h_prefix[n]);
  }
  if ((st = run_detect(c, n, p, max_oct, cap, s, measure, tile_mode, block_mask)) != CDVS_OK) return st;
  prof_end(c, 0, max_oct, ev, s);
  // the staged host images are read no more
  if (!(flags & CDVS_INPUT_DEVICE) && (e = cudaEventRecord(hset.in_free, s)) != cudaSuccess)
    return cuda_fail(c, e, "staging set");
  int* h_small = static_cast<int*>(c->hs().small.p);

  if (mode == kScaleSpace) {
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "scale space");
    return CDVS_OK;  // the caller copies the levels out
  }

  if (mode == kCandidates) {
    std::vector<int> counts(n);
    if ((e = cudaMemcpyAsync(counts.data(), c->cand_count.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(h_small, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(c, e, "candidate readback");
    int status_bits = h_small[0];
    if ((status_bits & kStatusCandOverflow) && !c->overflow_rerun) {
      // a queue overflowed: the call runs again with room for every
      // candidate, so no candidate is dropped in whatever order they came
      grow_cap_floor(c, counts.data(), n);
      c->overflow_rerun = true;
      st = run(c, mode, n, images, sizes, params, pin, kp_out, desc_out, capacity, kp_count, flags, caller_s);
      c->overflow_rerun = false;
      return st;
    }
    int written = 0;
    std::vector<Cand> tmp;
    for (int i = 0; i < n; ++i) {
      int m = std::min(counts[i], cap);
      const int room = std::max(0, capacity - written);
      if (m > room) {
        m = room;
        status_bits |= kStatusOutTruncated;
      }
      tmp.resize(m);
      if (m > 0 &&
          (e = cudaMemcpy(tmp.data(), static_cast<Cand*>(c->cands.p) + (size_t)i * cap, sizeof(Cand) * m,
                          cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, e, "candidate readback");
      for (int j = 0; j < m; ++j) {
        const Cand& q = tmp[j];
        const float sc = (float)(1 << q.octave);
        cdvs_keypoint& k = kp_out[written + j];
        k.x = q.xo * sc;
        k.y = q.yo * sc;
        k.sigma = q.so * sc;
        k.theta = 0.0f;
        k.response = q.resp;
        k.p_ss = q.pss;
        k.ratio = q.ratio;
        k.octave = q.octave;
        k.scale_idx = 0;
        k.type = q.type;
        k.reserved = 0;
        k.image = i;
        k.parent_id = -1;
      }
      kp_count[i] = m;
      written += m;
    }
    return map_status(c, status_bits);
  }

  if (mode == kExtract) {
    SelectArgs a;
    a.plans = static_cast<const ImgPlan*>(c->plans.p);
    a.cands = static_cast<const Cand*>(c->cands.p);
    a.cand_count = static_cast<const int*>(c->cand_count.p);
    a.cand_cap = cap;
    a.order = static_cast<int*>(c->order.p);
    a.keep = static_cast<unsigned char*>(c->keep.p);
    a.skey = static_cast<float4*>(c->skey.p);
    a.soct = static_cast<unsigned char*>(c->soct.p);
    a.sel = static_cast<Cand*>(c->sel.p);
    a.sel_count = static_cast<int*>(c->sel_count.p);
    a.N = N;
    a.dlog2 = p.dedupe_dlog2;
    a.status = static_cast<int*>(c->status.p);
    ev = prof_begin(c, s);
    if ((e = launch_select(a, n, s)) != cudaSuccess) return cuda_fail(c, e, "select launch");
    prof_end(c, 1, 1, ev, s);
  } else {  // kDescribe: the given points become the selected list
    std::vector<Cand> h_sel(slots);
    std::vector<int> h_cnt(n);
    for (int i = 0; i < n; ++i) {
      const int m = pin->counts[i];
      if (m < 0 || m > N) return fail(c, CDVS_INVALID_ARGUMENT, "n_pts[i] must be in 0..max_keypoints");
      h_cnt[i] = m;
      for (int j = 0; j < m; ++j) {
        const cdvs_keypoint& k = pin->pts[(size_t)i * pin->stride + j];
        if (k.octave < 0 || k.octave >= c->h_plans[i].n_oct)
          return fail(c, CDVS_INVALID_ARGUMENT, "point octave out of range");
        const float inv = 1.0f / (float)(1 << k.octave);
        Cand& q = h_sel[(size_t)i * N + j];
        q.xo = k.x * inv;
        q.yo = k.y * inv;
        q.so = k.sigma * inv;
        q.resp = k.response;
        q.pss = k.p_ss;
        q.ratio = k.ratio;
        q.octave = k.octave;
        q.type = k.type;
        q.spare = 0;
      }
    }
    if ((e = cudaMemcpyAsync(c->sel.p, h_sel.data(), sizeof(Cand) * slots, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(c->sel_count.p, h_cnt.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(c, e, "point upload");
  }

  DescribeArgs d = describe_args(c, n, p);
  d.kp_capacity = capacity;
  const bool dev_out = (flags & CDVS_OUTPUT_DEVICE) != 0;
  if (dev_out && (reinterpret_cast<uintptr_t>(desc_out) & 15) != 0)
    return fail(c, CDVS_INVALID_ARGUMENT, "device desc_out must be 16-byte aligned");
  if (dev_out) {
    d.kp_out = kp_out;
    d.desc_out = desc_out;
    d.kp_count = kp_count;
  } else {
    // the set's output copy, once the records it held two calls back are out
    if ((e = ensure(hset.out_kp, sizeof(cdvs_keypoint) * (size_t)capacity)) != cudaSuccess ||
        (e = ensure(hset.out_desc, sizeof(float) * 128 * (size_t)capacity)) != cudaSuccess ||
        (e = ensure(hset.out_count, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, hset.out_free, 0)) != cudaSuccess)
      return cuda_fail(c, e, "output staging");
    d.kp_out = static_cast<cdvs_keypoint*>(hset.out_kp.p);
    d.desc_out = static_cast<float*>(hset.out_desc.p);
    d.kp_count = static_cast<int*>(hset.out_count.p);
  }
  // Description and packing over the whole batch as one image group (the
  // kernels take a group's image range; returning host records per group
  // while later groups were described measured slower than one readback).
  const int groups = 1;
  if ((e = ensure(c->out_counters, sizeof(int) * (3 * kMaxOutGroups + 1))) != cudaSuccess ||
      (e = cudaMemsetAsync(c->out_counters.p, 0, sizeof(int) * (3 * kMaxOutGroups + 1), s)) != cudaSuccess)
    return cuda_fail(c, e, "output counters");
  unsigned* ctr = static_cast<unsigned*>(c->out_counters.p);
  int* bases = reinterpret_cast<int*>(ctr + 2 * kMaxOutGroups);
  for (int g = 0; g < groups; ++g) {
    d.img_begin = (int)((long long)n * g / groups);
    d.img_end = (int)((long long)n * (g + 1) / groups);
    d.claim = ctr + g;
    d.scan_done = ctr + kMaxOutGroups + g;
    d.base_in = bases + g;
    d.base_out = bases + g + 1;
    d.last_group = g == groups - 1;
    ev = prof_begin(c, s);
    if ((e = launch_describe(d, p.storage, c->n_sms, s)) != cudaSuccess) return cuda_fail(c, e, "describe launch");
    prof_end(c, 2, 1, ev, s);
    ev = prof_begin(c, s);
    if ((e = launch_pack(d, s)) != cudaSuccess) return cuda_fail(c, e, "packing launch");
    prof_end(c, 3, 1, ev, s);
    ev = prof_begin(c, s);
    if ((e = launch_copy(d, c->n_sms, s)) != cudaSuccess) return cuda_fail(c, e, "copy launch");
    prof_end(c, 4, 1, ev, s);
  }
  if ((!async || !dev_out) &&
      ((e = cudaMemcpyAsync(h_small, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
       (e = cudaMemcpyAsync(h_small + 1, c->rec_total.p, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
       (!dev_out && (e = cudaEventRecord(hset.packed, s)) != cudaSuccess)))
    return cuda_fail(c, e, "status readback");
  if (graph) {
    cudaGraph_t g = nullptr;
    capture.on = false;
    if ((e = cudaStreamEndCapture(s, &g)) != cudaSuccess) return cuda_fail(c, e, "graph capture");
    if (c->gexec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(c->gexec, g, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
    }
    if (!c->gexec && (e = cudaGraphInstantiate(&c->gexec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(c, e, "graph instantiation");
    }
    cudaGraphDestroy(g);
    if ((e = cudaGraphLaunch(c->gexec, s)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
    if (s != caller_s) {  // the caller's stream continues after the graph
      if ((e = cudaEventRecord(c->gev, s)) != cudaSuccess || (e = cudaStreamWaitEvent(caller_s, c->gev, 0)) != cudaSuccess)
        return cuda_fail(c, e, "graph stream");
    }
  }
  if (async) {  // the caller synchronizes; cdvs_wait reports the status bits
    c->async_open = true;
    if (!dev_out) {
      // the previous call's records go out now (this call's work is already
      // queued behind it); this call's go out at the next call or cdvs_wait
      if ((st = flush_readback(c)) != CDVS_OK) return st;
      c->pend = PendingReadback{true, c->cur_set, n, kp_out, desc_out, kp_count};
    }
    c->err.clear();
    return CDVS_OK;
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "status readback");
  const int status_bits = h_small[0];
  const int total = h_small[1];
  if ((status_bits & kStatusCandOverflow) && !c->overflow_rerun && mode == kExtract) {
    // a queue overflowed: the call runs again with room for every candidate,
    // so the result never depends on which candidates came first
    std::vector<int> counts(n);
    if ((e = cudaMemcpy(counts.data(), c->cand_count.p, sizeof(int) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(c, e, "candidate counts");
    grow_cap_floor(c, counts.data(), n);
    c->overflow_rerun = true;
    st = run(c, mode, n, images, sizes, params, pin, kp_out, desc_out, capacity, kp_count, flags, caller_s);
    c->overflow_rerun = false;
    return st;
  }
  if (!dev_out) {
    if ((e = cudaMemcpyAsync(kp_count, hset.out_count.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (total > 0 && (e = cudaMemcpyAsync(kp_out, hset.out_kp.p, sizeof(cdvs_keypoint) * (size_t)total,
                                           cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
        (total > 0 && (e = cudaMemcpyAsync(desc_out, hset.out_desc.p, sizeof(float) * 128 * (size_t)total,
                                           cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(c, e, "output readback");
  }
  return map_status(c, status_bits);
}

}  // namespace

extern "C" {

void cdvs_params_default(cdvs_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->num_octaves = 4;
  p->scales_per_octave = 4;
  p->sigma0 = 1.6f;
  p->sigma_in = 0.5f;
  p->contrast_T = 4.0f;
  p->edge_r = 10.0f;
  p->offset_max = 0.5f;
  p->ori_radius = 3.96f;     // Sec. IV-B
  p->ori_peak_ratio = 0.8f;  // Sec. IV-B
  p->ori_weight_sigma = 1.5f;
  p->desc_radius = 6.0f;     // Alg. 2 stage B
  p->cell_side = 3.0f;       // Sec. IV-B
  p->desc_weight_sigma = 2.0f;
  p->dedupe_dlog2 = 1.0f / 3.0f;
  p->max_keypoints = 300;    // Sec. III-B
  p->max_orientations = 4;
  p->upright = 0;
  p->storage = CDVS_STORAGE_FP32;
  p->use_proposal = 0;
  p->proposal_threshold = 0.5f;
  p->max_side = 0;
}

cdvs_status cdvs_create(cdvs_ctx** out, int device, size_t workspace_bytes_hint) {
  if (!out) return CDVS_INVALID_ARGUMENT;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return CDVS_CUDA_ERROR;
  }
  if (device < 0 || device >= ndev) return CDVS_INVALID_ARGUMENT;
  if (cudaSetDevice(device) != cudaSuccess) return CDVS_CUDA_ERROR;
  cdvs_ctx* c = new cdvs_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device);
  if (workspace_bytes_hint > 0 && ensure(c->levels, workspace_bytes_hint) != cudaSuccess) {
    delete c;
    return CDVS_OUT_OF_MEMORY;
  }
  *out = c;
  return CDVS_OK;
}

void cdvs_destroy(cdvs_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  DevBuf* bufs[] = {&c->levels,  &c->cands,   &c->cand_count, &c->order,   &c->keep, &c->skey, &c->soct,
                    &c->sel,     &c->sel_count, &c->ori_theta, &c->ori_count, &c->rec_off,
                    &c->rec_total, &c->plans,
                    &c->tile_prefix, &c->status, &c->input, &c->dump, &c->stage_kp, &c->stage_desc,
                    &c->prop_theta, &c->prop_imgs, &c->prop_logits, &c->prop_mode, &c->prop_ws,
                    &c->resized, &c->resize_jobs, &c->scfv_model, &c->scfv_desc, &c->scfv_q,
                    &c->scfv_out, &c->scfv_off, &c->out_counters};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->d2h_stream) {
    cudaStreamSynchronize(c->d2h_stream);
    cudaStreamDestroy(c->d2h_stream);
  }
  for (StageSet& hs : c->hset) {
    for (HostBuf* h : {&hs.plans, &hs.prefix, &hs.prop, &hs.jobs, &hs.plans2, &hs.small})
      if (h->p) cudaFreeHost(h->p);
    for (DevBuf* b : {&hs.input, &hs.out_kp, &hs.out_desc, &hs.out_count})
      if (b->p) cudaFree(b->p);
    for (cudaEvent_t ev : {hs.done, hs.in_free, hs.out_free, hs.packed})
      if (ev) cudaEventDestroy(ev);
  }
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->gev) cudaEventDestroy(c->gev);
  for (const ProfRec& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (const auto& m : c->measures) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    for (cudaEvent_t e : c->ready) cudaEventDestroy(e);
    cudaStreamDestroy(c->copy_stream);
  }
  delete c;
}

const char* cdvs_last_error(const cdvs_ctx* c) { return c ? c->err.c_str() : "null context"; }

cdvs_status cdvs_extract(cdvs_ctx* c, int32_t n_images, const uint8_t* const* images,
                         const cdvs_image_desc* sizes, const cdvs_params* params, cdvs_keypoint* kp_out,
                         float* desc_out, int32_t kp_capacity, int32_t* kp_count, uint32_t flags,
                         void* cuda_stream) {
  return run(c, kExtract, n_images, images, sizes, params, nullptr, kp_out, desc_out, kp_capacity, kp_count,
             flags, static_cast<cudaStream_t>(cuda_stream));
}

cdvs_status cdvs_candidates(cdvs_ctx* c, int32_t n_images, const uint8_t* const* images,
                            const cdvs_image_desc* sizes, const cdvs_params* params, cdvs_keypoint* cand_out,
                            int32_t cand_capacity, int32_t* cand_count, uint32_t flags, void* cuda_stream) {
  return run(c, kCandidates, n_images, images, sizes, params, nullptr, cand_out, nullptr, cand_capacity,
             cand_count, flags, static_cast<cudaStream_t>(cuda_stream));
}

cdvs_status cdvs_describe(cdvs_ctx* c, int32_t n_images, const uint8_t* const* images,
                          const cdvs_image_desc* sizes, const cdvs_params* params, const cdvs_keypoint* pts,
                          const int32_t* n_pts, int32_t pts_stride, cdvs_keypoint* kp_out, float* desc_out,
                          int32_t kp_capacity, int32_t* kp_count, uint32_t flags, void* cuda_stream) {
  if (!pts || !n_pts || pts_stride < 0) return fail(c, CDVS_INVALID_ARGUMENT, "points are NULL");
  if (flags & CDVS_INPUT_DEVICE) {
    // point lists are read on the host by this entry point
  }
  PointsIn pin{pts, n_pts, pts_stride};
  return run(c, kDescribe, n_images, images, sizes, params, &pin, kp_out, desc_out, kp_capacity, kp_count,
             flags, static_cast<cudaStream_t>(cuda_stream));
}

cdvs_status cdvs_dedupe_select(cdvs_ctx* c, int32_t n, const cdvs_image_desc* sizes, const cdvs_keypoint* cand,
                               const int32_t* cand_count, int32_t cand_stride, const cdvs_params* params,
                               cdvs_keypoint* sel_out, int32_t sel_capacity, int32_t* sel_count, uint32_t flags,
                               void* cuda_stream) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  cdvs_status st = check_params(c, params);
  if (st != CDVS_OK) return st;
  if (c->async_open) return fail(c, CDVS_INVALID_ARGUMENT, "asynchronous extractions are pending: call cdvs_wait first");
  if (n < 0 || !sizes || (n > 0 && (!cand || !cand_count || !sel_out || !sel_count)))
    return fail(c, CDVS_INVALID_ARGUMENT, "NULL argument or n < 0");
  if (flags & (CDVS_INPUT_DEVICE | CDVS_OUTPUT_DEVICE))
    return fail(c, CDVS_INVALID_ARGUMENT, "cdvs_dedupe_select takes host buffers only");
  if (n == 0) return CDVS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  const cdvs_params& p = *params;
  long long level_elems, max_pixels;
  int max_oct;
  if ((st = plan_batch(c, n, sizes, p, level_elems, max_oct, max_pixels)) != CDVS_OK) return st;
  int cap = 1;
  for (int i = 0; i < n; ++i) cap = std::max(cap, (int)cand_count[i]);
  const int N = p.max_keypoints;
  std::vector<Cand> h((size_t)n * cap);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < cand_count[i]; ++j) {
      const cdvs_keypoint& k = cand[(size_t)i * cand_stride + j];
      if (k.octave < 0 || k.octave >= c->h_plans[i].n_oct)
        return fail(c, CDVS_INVALID_ARGUMENT, "candidate octave is not one of the image's octaves");
      const float inv = 1.0f / (float)(1 << k.octave);
      Cand& q = h[(size_t)i * cap + j];
      q.xo = k.x * inv;
      q.yo = k.y * inv;
      q.so = k.sigma * inv;
      q.resp = k.response;
      q.pss = k.p_ss;
      q.ratio = k.ratio;
      q.octave = k.octave;
      q.type = k.type;
      q.spare = j;
    }
  if ((e = ensure(c->cands, sizeof(Cand) * h.size())) != cudaSuccess ||
      (e = ensure(c->cand_count, sizeof(int) * n)) != cudaSuccess ||
      (e = ensure(c->order, sizeof(int) * h.size())) != cudaSuccess || (e = ensure(c->keep, h.size())) != cudaSuccess ||
      (e = ensure(c->skey, sizeof(float4) * h.size())) != cudaSuccess || (e = ensure(c->soct, h.size())) != cudaSuccess ||
      (e = ensure(c->sel, sizeof(Cand) * (size_t)n * N)) != cudaSuccess ||
      (e = ensure(c->sel_count, sizeof(int) * n)) != cudaSuccess ||
      (e = ensure(c->status, sizeof(int) * 4)) != cudaSuccess ||
      (e = ensure(c->plans, sizeof(ImgPlan) * n)) != cudaSuccess)
    return cuda_fail(c, e, "workspace");
  std::vector<int> cnt(cand_count, cand_count + n);
  if ((e = cudaMemcpyAsync(c->cands.p, h.data(), sizeof(Cand) * h.size(), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(c->cand_count.p, cnt.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(c->plans.p, c->h_plans.data(), sizeof(ImgPlan) * n, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(c->status.p, 0, sizeof(int) * 4, s)) != cudaSuccess)
    return cuda_fail(c, e, "upload");
  SelectArgs a;
  a.plans = static_cast<const ImgPlan*>(c->plans.p);
  a.cands = static_cast<const Cand*>(c->cands.p);
  a.cand_count = static_cast<const int*>(c->cand_count.p);
  a.cand_cap = cap;
  a.order = static_cast<int*>(c->order.p);
  a.keep = static_cast<unsigned char*>(c->keep.p);
  a.skey = static_cast<float4*>(c->skey.p);
  a.soct = static_cast<unsigned char*>(c->soct.p);
  a.sel = static_cast<Cand*>(c->sel.p);
  a.sel_count = static_cast<int*>(c->sel_count.p);
  a.N = N;
  a.dlog2 = p.dedupe_dlog2;
  a.status = static_cast<int*>(c->status.p);
  if ((e = launch_select(a, n, s)) != cudaSuccess) return cuda_fail(c, e, "select launch");
  std::vector<Cand> hs((size_t)n * N);
  std::vector<int> hc(n);
  int status_bits = 0;
  if ((e = cudaMemcpyAsync(hs.data(), c->sel.p, sizeof(Cand) * hs.size(), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(hc.data(), c->sel_count.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&status_bits, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(c, e, "readback");
  int written = 0;
  for (int i = 0; i < n; ++i) {
    int m = hc[i];
    if (written + m > sel_capacity) {
      m = std::max(0, sel_capacity - written);
      status_bits |= kStatusOutTruncated;
    }
    for (int r = 0; r < m; ++r) {
      const Cand& q = hs[(size_t)i * N + r];
      const float sc = (float)(1 << q.octave);
      cdvs_keypoint& k = sel_out[written + r];
      k.x = q.xo * sc;
      k.y = q.yo * sc;
      k.sigma = q.so * sc;
      k.theta = 0.0f;
      k.response = q.resp;
      k.p_ss = q.pss;
      k.ratio = q.ratio;
      k.octave = q.octave;
      k.scale_idx = 0;
      k.type = q.type;
      k.reserved = 0;
      k.image = i;
      k.parent_id = q.spare;  // index of the point in the caller's list
    }
    sel_count[i] = m;
    written += m;
  }
  return map_status(c, status_bits);
}

cdvs_status cdvs_scale_space(cdvs_ctx* c, const uint8_t* image, const cdvs_image_desc* size,
                             const cdvs_params* params, float* levels_out, size_t capacity, int32_t* n_octaves,
                             uint32_t flags, void* cuda_stream) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (!image || !size || !levels_out || !n_octaves) return fail(c, CDVS_INVALID_ARGUMENT, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const uint8_t* imgs[1] = {image};
  cdvs_status st = run(c, kScaleSpace, 1, imgs, size, params, nullptr, nullptr, nullptr, 0, nullptr,
                       flags & CDVS_INPUT_DEVICE, s);
  if (st != CDVS_OK) return st;
  const ImgPlan& P = c->h_plans[0];
  size_t need = 0;
  for (int o = 0; o < P.n_oct; ++o) need += (size_t)kScales * P.oct[o].W * P.oct[o].H;
  if (need > capacity) return fail(c, CDVS_INVALID_ARGUMENT, "levels_out capacity too small");
  cudaError_t e;
  float* dst = levels_out;
  if (!(flags & CDVS_OUTPUT_DEVICE)) {
    if ((e = ensure(c->dump, need * sizeof(float))) != cudaSuccess) return cuda_fail(c, e, "dump buffer");
    dst = static_cast<float*>(c->dump.p);
  }
  size_t off = 0;
  for (int o = 0; o < P.n_oct; ++o)
    for (int k = 0; k < kScales; ++k) {
      const OctPlan& op = P.oct[o];
      if ((e = launch_levels_to_f32(c->levels.p, params->storage, op.W, op.H, op.tr,
                                    op.level_off + (long long)k * op.lpitch * op.H, op.lpitch, dst + off, s)) !=
          cudaSuccess)
        return cuda_fail(c, e, "level copy");
      off += (size_t)op.W * op.H;
    }
  if (!(flags & CDVS_OUTPUT_DEVICE)) {
    if ((e = cudaMemcpyAsync(levels_out, dst, need * sizeof(float), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(c, e, "level readback");
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "sync");
  *n_octaves = P.n_oct;
  return CDVS_OK;
}

cdvs_status cdvs_wait(cdvs_ctx* c, void* cuda_stream) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (!c->async_open) {
    c->err.clear();
    return CDVS_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  cdvs_status st = flush_readback(c);
  if (st != CDVS_OK) return st;
  if (c->d2h_stream && (e = cudaStreamSynchronize(c->d2h_stream)) != cudaSuccess) return cuda_fail(c, e, "readback");
  HostBuf& h = c->hs().small;
  if ((e = ensure_host(h, sizeof(int) * (4 + kMaxOutGroups + 1))) != cudaSuccess ||
      (e = cudaMemcpyAsync(h.p, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(c, e, "status readback");
  c->async_open = false;
  const int bits = static_cast<int*>(h.p)[0];
  // an asynchronous call cannot be run again: its truncation is reported,
  // and later calls get twice the capacity
  if (bits & kStatusCandOverflow) c->cap_floor = std::max(c->cap_floor, 2 * c->last_cap);
  return map_status(c, bits);
}

cdvs_status cdvs_set_detect_variant(cdvs_ctx* c, int32_t variant) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (variant < -1 || variant >= kDetectVariants)
    return fail(c, CDVS_INVALID_ARGUMENT, "variant must be -1 (tuned) or 0..3");
  c->variant_mode = variant;
  return CDVS_OK;
}

int32_t cdvs_detect_tuning(cdvs_ctx* c, char* buf, int32_t capacity) {
  if (!c) return -1;
  cudaSetDevice(c->device);
  harvest_measures(c);
  std::string j = "{\"mode\": " + std::to_string(c->variant_mode) + ", \"variants\": [";
  for (int v = 0; v < kDetectVariants; ++v)
    j += std::string(v ? ", " : "") + "\"" + detect_variant_name(v) + "\"";
  j += "], \"classes\": [";
  for (size_t i = 0; i < c->tune.size(); ++i) {
    const auto& t = c->tune[i];
    j += std::string(i ? ", " : "") + "{\"octaves\": \"" + (t.later ? "1+" : "0") + "\", \"storage\": \"" +
         (t.storage == CDVS_STORAGE_FP16 ? "fp16" : "fp32") + "\", \"radii\": [";
    for (int k = 0; k < kScales; ++k) j += std::string(k ? ", " : "") + std::to_string(t.radii[k]);
    j += "], \"us_per_tile\": [";
    for (int v = 0; v < kDetectVariants; ++v) {
      char num[32];
      if (t.ms_per_tile[v] < 0.0f) std::snprintf(num, sizeof(num), "null");
      else std::snprintf(num, sizeof(num), "%.4f", 1e3 * t.ms_per_tile[v]);
      j += std::string(v ? ", " : "") + num;
    }
    j += std::string("], \"tuned\": ") + (class_tuned(t) ? "true" : "false") + "}";
  }
  j += "], \"last_call_variants\": [";
  for (int o = 0; o < kMaxOctaves; ++o) j += std::string(o ? ", " : "") + std::to_string(c->oct_variant[o]);
  j += "]}";
  if (buf && capacity > 0) {
    const size_t m = std::min((size_t)capacity - 1, j.size());
    std::memcpy(buf, j.data(), m);
    buf[m] = 0;
  }
  return (int32_t)j.size();
}

cdvs_status cdvs_set_candidate_capacity(cdvs_ctx* c, int32_t per_image) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (per_image < 0 || per_image > (1 << 22)) return fail(c, CDVS_INVALID_ARGUMENT, "per_image must be in 0..2^22");
  c->cap_fixed = per_image;
  c->cap_floor = 0;
  return CDVS_OK;
}

void cdvs_inject_alloc_failures(int32_t count) { g_fail_allocs.store(count > 0 ? count : 0); }

void cdvs_inject_scfv_wait_timeouts(int32_t count) { g_skip_products.store(count > 0 ? count : 0); }

cdvs_status cdvs_profile(cdvs_ctx* c, int32_t enable) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  c->prof = enable != 0;
  return CDVS_OK;
}

cdvs_status cdvs_set_scfv_model(cdvs_ctx* c, const cdvs_scfv_model* m) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (!m || !m->pca_mean || !m->pca || !m->weights || !m->means || !m->variances)
    return fail(c, CDVS_INVALID_ARGUMENT, "NULL model array");
  std::vector<float> d(kScfvModelFloats);
  std::vector<__half> bh(2 * kScfvWHalfWords), bl(2 * kScfvWHalfWords);  // the B operand's halves
  // the gradient products take [1 | y | y^2] in FP16 halves: bounded PCA
  // rows (orthonormal ones have norm 1) and mean keep |y| <= 2 * 64 for unit
  // descriptors, so y^2 stays far inside FP16's range
  double mean2 = 0.0;
  for (int k = 0; k < 128; ++k) mean2 += (double)m->pca_mean[k] * m->pca_mean[k];
  if (!(mean2 <= 4.0)) return fail(c, CDVS_INVALID_ARGUMENT, "the PCA mean must have norm <= 2");
  for (int j = 0; j < kScfvDim; ++j) {
    double r2 = 0.0;
    for (int k = 0; k < 128; ++k) r2 += (double)m->pca[j * 128 + k] * m->pca[j * 128 + k];
    if (!(r2 <= 64.0 * 64.0)) return fail(c, CDVS_INVALID_ARGUMENT, "PCA rows must have norm <= 64");
  }
  for (int k = 0; k < 128; ++k) {
    d[kScfvOffMean + k] = m->pca_mean[k];
    for (int j = 0; j < kScfvDim; ++j) d[kScfvOffPcaT + k * kScfvDim + j] = m->pca[j * 128 + k];
  }
  for (int i = 0; i < kScfvComp; ++i) {
    const double w = m->weights[i];
    if (!(w > 0.0)) return fail(c, CDVS_INVALID_ARGUMENT, "GMM weights must be positive");
    double logdet = 0.0;
    for (int k = 0; k < kScfvDim; ++k) {
      const double v = m->variances[i * kScfvDim + k];
      if (!(v > 0.0)) return fail(c, CDVS_INVALID_ARGUMENT, "GMM variances must be positive");
      d[kScfvOffMu + i * kScfvDim + k] = m->means[i * kScfvDim + k];
      d[kScfvOffIsd + i * kScfvDim + k] = (float)(1.0 / std::sqrt(v));
      logdet += std::log(2.0 * 3.14159265358979323846 * v);
    }
    d[kScfvOffLw + i] = (float)(std::log(w) - 0.5 * logdet);
    d[kScfvOffNmu + i] = (float)(1.0 / std::sqrt(w));
    d[kScfvOffNsig + i] = (float)(1.0 / std::sqrt(2.0 * w));
    // Eq. 10's matrix form: -1/2 sum_k (y_k - mu_k)^2 / v_k
    //   = sum_k y_k^2 (-1/(2 v_k)) + sum_k y_k (mu_k / v_k) - 1/2 sum_k mu_k^2 / v_k
    double cq = 0.0, col[2 * kScfvDim], big = 0.0;
    for (int k = 0; k < kScfvDim; ++k) {
      const double v = m->variances[i * kScfvDim + k], mu = m->means[i * kScfvDim + k];
      col[k] = -0.5 / v;
      col[kScfvDim + k] = mu / v;
      cq += mu * mu / v;
    }
    for (double x : col) big = std::max(big, std::fabs(x));
    if (!std::isfinite(big) || !std::isfinite(cq)) return fail(c, CDVS_INVALID_ARGUMENT, "GMM parameters overflow");
    // column i scaled by a power of two, largest |entry| <= 2^14, then split
    // into FP16 halves (the lo half carries the next 11 bits)
    const int ex = big > 0.0 ? 14 - (int)std::ceil(std::log2(big)) : 0;
    for (int k = 0; k < 2 * kScfvDim; ++k) {
      const double x = std::ldexp(col[k], ex);
      const __half h = __float2half_rn((float)x);
      bh[kScfvTcBIndex(i, k)] = h;
      bl[kScfvTcBIndex(i, k)] = __float2half_rn((float)(x - (double)__half2float(h)));
    }
    d[kScfvOffInvE + i] = (float)std::ldexp(1.0, -ex);
    d[kScfvOffC + i] = (float)(std::log(w) - 0.5 * logdet - 0.5 * cq);
  }
  std::memcpy(d.data() + kScfvOffW, bh.data(), sizeof(__half) * bh.size());
  std::memcpy(d.data() + kScfvOffW + kScfvWHalfWords, bl.data(), sizeof(__half) * bl.size());
  // P^T as FP16 hi / lo B fragments of the projection (|P| <= 64 by the row
  // norm check above)
  {
    uint32_t* pf = reinterpret_cast<uint32_t*>(d.data() + kScfvOffPf);
    for (int st = 0; st < 128 / 16; ++st)
      for (int j8 = 0; j8 < kScfvDim / 8; ++j8)
        for (int lane = 0; lane < 32; ++lane)
          for (int q = 0; q < 2; ++q) {
            const int g = lane / 4, t = lane % 4, k0 = 16 * st + 2 * t + 8 * q, j = 8 * j8 + g;
            __half hi[2], lo[2];
            for (int e = 0; e < 2; ++e) {
              const float x = m->pca[j * 128 + k0 + e];
              hi[e] = __float2half_rn(x);
              lo[e] = __float2half_rn(x - __half2float(hi[e]));
            }
            const int idx = kScfvPfIndex(st, j8, lane, q);
            std::memcpy(pf + idx, hi, 4);
            std::memcpy(pf + 2048 + idx, lo, 4);
          }
  }
  cudaError_t e;
  if ((e = cudaSetDevice(c->device)) != cudaSuccess || (e = ensure(c->scfv_model, sizeof(float) * d.size())) != cudaSuccess ||
      (e = cudaMemcpy(c->scfv_model.p, d.data(), sizeof(float) * d.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(c, e, "SCFV model");
  c->scfv_set = true;
  return CDVS_OK;
}

cdvs_status cdvs_scfv(cdvs_ctx* c, int32_t n, const float* desc, const int32_t* counts, int32_t n_select,
                      float* g_mu, float* g_sigma, float* delta, int32_t* order, uint32_t* bits, uint32_t flags,
                      void* cuda_stream) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (!c->scfv_set) return fail(c, CDVS_INVALID_ARGUMENT, "no cdvs_set_scfv_model call");
  if (n < 0 || n > kMaxBatch || n_select < 0 || n_select > kScfvComp)
    return fail(c, CDVS_INVALID_ARGUMENT, "n_images in 0..4096 and n_select in 0..512 required");
  if (n == 0) return CDVS_OK;
  if (!counts || (n_select > 0 && !bits)) return fail(c, CDVS_INVALID_ARGUMENT, "NULL counts or bits");
  std::vector<int> off(n + 2, 0);  // record offsets, then the device status word (0)
  for (int i = 0; i < n; ++i) {
    if (counts[i] < 0) return fail(c, CDVS_INVALID_ARGUMENT, "negative count");
    off[i + 1] = off[i] + counts[i];
  }
  const int n_rec = off[n];
  if (n_rec > 0 && !desc) return fail(c, CDVS_INVALID_ARGUMENT, "NULL desc");
  const bool dev_in = (flags & CDVS_INPUT_DEVICE) != 0, dev_out = (flags & CDVS_OUTPUT_DEVICE) != 0;
  if (dev_in && (reinterpret_cast<uintptr_t>(desc) & 15) != 0)
    return fail(c, CDVS_INVALID_ARGUMENT, "device desc must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  if ((e = cudaSetDevice(c->device)) != cudaSuccess) return cuda_fail(c, e, "device");
  const size_t per = (size_t)kScfvComp * kScfvDim;
  // scratch: projected descriptors, posteriors, and the outputs the caller
  // does not take (or takes on the host)
  const size_t out_floats = (size_t)n * (2 * per + kScfvComp) + (size_t)n * kScfvComp + (size_t)n * kScfvComp;
  if ((e = ensure(c->scfv_q, std::max<size_t>(scfv_ops_bytes(n_rec), 16))) != cudaSuccess ||
      (e = ensure(c->scfv_out, sizeof(float) * out_floats)) != cudaSuccess ||
      (e = ensure(c->scfv_off, sizeof(int) * (n + 2))) != cudaSuccess ||
      (!dev_in && n_rec > 0 && (e = ensure(c->scfv_desc, sizeof(float) * 128 * (size_t)n_rec)) != cudaSuccess))
    return cuda_fail(c, e, "SCFV workspace");
  float* sc = static_cast<float*>(c->scfv_out.p);
  float* s_mu = sc;
  float* s_sig = s_mu + (size_t)n * per;
  float* s_delta = s_sig + (size_t)n * per;
  int* s_order = reinterpret_cast<int*>(s_delta + (size_t)n * kScfvComp);
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(s_order + (size_t)n * kScfvComp);
  float* o_mu = dev_out && g_mu ? g_mu : s_mu;
  float* o_sig = dev_out && g_sigma ? g_sigma : s_sig;
  float* o_delta = dev_out && delta ? delta : s_delta;
  int* o_order = dev_out && order ? order : s_order;
  uint32_t* o_bits = dev_out && bits ? bits : s_bits;
  const float* d_desc = desc;
  if (!dev_in && n_rec > 0) {
    if ((e = cudaMemcpyAsync(c->scfv_desc.p, desc, sizeof(float) * 128 * (size_t)n_rec, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return cuda_fail(c, e, "descriptor upload");
    d_desc = static_cast<const float*>(c->scfv_desc.p);
  }
  int* d_status = static_cast<int*>(c->scfv_off.p) + n + 1;
  int skip = 0;  // the testing hook: leave one call's tensor-core products unissued
  for (int f = g_skip_products.load(); f > 0;)
    if (g_skip_products.compare_exchange_weak(f, f - 1)) {
      skip = 1;
      break;
    }
  if ((e = cudaMemcpyAsync(c->scfv_off.p, off.data(), sizeof(int) * (n + 2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = launch_scfv(d_desc, n_rec, static_cast<const int*>(c->scfv_off.p), n,
                       static_cast<const float*>(c->scfv_model.p), n_select, c->scfv_q.p, o_mu, o_sig, o_delta,
                       o_order, o_bits, d_status, skip,
                       c->n_sms, s)) != cudaSuccess)
    return cuda_fail(c, e, "SCFV launch");
  if (!dev_out) {
    struct Out {
      void* h;
      const void* d;
      size_t bytes;
    } outs[] = {{g_mu, o_mu, sizeof(float) * n * per}, {g_sigma, o_sig, sizeof(float) * n * per},
                {delta, o_delta, sizeof(float) * n * kScfvComp}, {order, o_order, sizeof(int) * n * kScfvComp},
                {bits, o_bits, sizeof(uint32_t) * (size_t)n * n_select}};
    for (const Out& o : outs)
      if (o.h && o.bytes && (e = cudaMemcpyAsync(o.h, o.d, o.bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(c, e, "SCFV readback");
  }
  if (!dev_in || !dev_out) {
    int st = 0;
    if ((e = cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(c, e, "SCFV");
    if (st & kStatusTimeout)
      return fail(c, CDVS_DEVICE_TIMEOUT, "SCFV: the tensor-core products did not complete within the bounded wait");
  }
  return CDVS_OK;
}

cdvs_status cdvs_probe_fp32_rate(cdvs_ctx* c, double* tflops) {
  if (!c || !tflops) return CDVS_INVALID_ARGUMENT;
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess) e = probe_ffma2(c->n_sms, tflops);
  if (e != cudaSuccess) return cuda_fail(c, e, "FP32 rate probe");
  return CDVS_OK;
}

cdvs_status cdvs_set_graph(cdvs_ctx* c, int32_t enable) {
  if (!c || (enable != 0 && enable != 1)) return CDVS_INVALID_ARGUMENT;
  if (c->async_open) return fail(c, CDVS_INVALID_ARGUMENT, "asynchronous extractions are pending: call cdvs_wait first");
  c->graph = enable != 0;
  if (!c->graph && c->gexec) {
    cudaSetDevice(c->device);
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return CDVS_OK;
}

cdvs_status cdvs_resize(cdvs_ctx* c, int32_t n, const uint8_t* const* images, const cdvs_image_desc* sizes,
                        int32_t max_side, uint8_t* out, size_t capacity, cdvs_image_desc* out_sizes, uint32_t flags,
                        void* cuda_stream) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (c->async_open) return fail(c, CDVS_INVALID_ARGUMENT, "asynchronous extractions are pending: call cdvs_wait first");
  if (n < 0 || n > kMaxBatch) return fail(c, CDVS_INVALID_ARGUMENT, "n_images must be in 0..4096");
  if (n == 0) return CDVS_OK;
  if (!images || !sizes || !out || !out_sizes) return fail(c, CDVS_INVALID_ARGUMENT, "NULL argument");
  if (max_side < 0 || max_side > 32768) return fail(c, CDVS_INVALID_ARGUMENT, "max_side must be 0..32768");
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    if (!images[i]) return fail(c, CDVS_INVALID_ARGUMENT, "image pointer is NULL");
    if (sizes[i].width < 1 || sizes[i].height < 1 || sizes[i].width > 32768 || sizes[i].height > 32768 ||
        sizes[i].pitch_bytes < sizes[i].width)
      return fail(c, CDVS_UNSUPPORTED_SIZE, "image sizes must be 1..32768 with pitch >= width");
    int W2, H2;
    resize_target(sizes[i].width, sizes[i].height, max_side, W2, H2);
    out_sizes[i].width = W2;
    out_sizes[i].height = H2;
    out_sizes[i].pitch_bytes = W2;
    need += (size_t)W2 * H2;
  }
  if (need > capacity) return fail(c, CDVS_UNSUPPORTED_SIZE, "out too small");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  if ((e = cudaSetDevice(c->device)) != cudaSuccess) return cuda_fail(c, e, "device");
  // inputs on the device (staged when on the host)
  std::vector<const uint8_t*> src(images, images + n);
  if (!(flags & CDVS_INPUT_DEVICE)) {
    size_t total = 0;
    std::vector<size_t> off(n);
    for (int i = 0; i < n; ++i) {
      off[i] = total;
      total += ((size_t)sizes[i].pitch_bytes * sizes[i].height + 255) & ~(size_t)255;
    }
    if ((e = ensure(c->input, total)) != cudaSuccess) return cuda_fail(c, e, "input staging");
    for (int i = 0; i < n; ++i) {
      src[i] = static_cast<uint8_t*>(c->input.p) + off[i];
      if ((e = cudaMemcpyAsync(const_cast<uint8_t*>(src[i]), images[i], (size_t)sizes[i].pitch_bytes * sizes[i].height,
                               cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(c, e, "image upload");
    }
  }
  const bool dev_out = (flags & CDVS_OUTPUT_DEVICE) != 0;
  if (!dev_out && (e = ensure(c->resized, need)) != cudaSuccess) return cuda_fail(c, e, "output staging");
  uint8_t* dst = dev_out ? out : static_cast<uint8_t*>(c->resized.p);
  std::vector<ResizeJob> jobs;
  size_t o = 0;
  int max_pixels = 0;
  for (int i = 0; i < n; ++i) {
    const int W2 = out_sizes[i].width, H2 = out_sizes[i].height;
    if (W2 == sizes[i].width && H2 == sizes[i].height) {
      if ((e = cudaMemcpy2DAsync(dst + o, W2, src[i], sizes[i].pitch_bytes, W2, H2, cudaMemcpyDeviceToDevice, s)) !=
          cudaSuccess)
        return cuda_fail(c, e, "copy");
    } else {
      jobs.push_back(ResizeJob{src[i], sizes[i].width, sizes[i].height, sizes[i].pitch_bytes, dst + o, W2, H2, W2});
      max_pixels = std::max(max_pixels, H2);  // rows
    }
    o += (size_t)W2 * H2;
  }
  if (!jobs.empty() &&
      ((e = ensure(c->resize_jobs, sizeof(ResizeJob) * jobs.size())) != cudaSuccess ||
       (e = cudaMemcpyAsync(c->resize_jobs.p, jobs.data(), sizeof(ResizeJob) * jobs.size(), cudaMemcpyHostToDevice,
                            s)) != cudaSuccess ||
       (e = launch_resize(static_cast<const ResizeJob*>(c->resize_jobs.p), (int)jobs.size(), max_pixels, s)) !=
           cudaSuccess))
    return cuda_fail(c, e, "resize");
  if (!dev_out && (e = cudaMemcpyAsync(out, dst, need, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(c, e, "readback");
  if ((!dev_out || !(flags & CDVS_INPUT_DEVICE)) && (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(c, e, "resize");
  return CDVS_OK;
}

cdvs_status cdvs_set_proposal(cdvs_ctx* c, const float* params, int32_t n_params) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (c->async_open) return fail(c, CDVS_INVALID_ARGUMENT, "asynchronous extractions are pending: call cdvs_wait first");
  if (!params || n_params != kPropParams) return fail(c, CDVS_INVALID_ARGUMENT, "need CDVS_PROPOSAL_PARAMS floats");
  cudaError_t e;
  // the parameters, then the tensor-core B fragments of conv2 and conv3
  std::vector<uint32_t> frag(kPropFragWords);
  pack_proposal_fragments(params, frag.data());
  const size_t pbytes = (sizeof(float) * kPropParams + 255) & ~(size_t)255;
  if ((e = cudaSetDevice(c->device)) != cudaSuccess ||
      (e = ensure(c->prop_theta, pbytes + sizeof(uint32_t) * kPropFragWords)) != cudaSuccess ||
      (e = cudaMemcpy(c->prop_theta.p, params, sizeof(float) * kPropParams, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(static_cast<uint8_t*>(c->prop_theta.p) + pbytes, frag.data(), sizeof(uint32_t) * kPropFragWords,
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(c, e, "proposal parameters");
  c->prop_set = true;
  return CDVS_OK;
}

cdvs_status cdvs_proposal_logits(cdvs_ctx* c, int32_t n, const uint8_t* const* images, const cdvs_image_desc* sizes,
                                 float* logits_out, int32_t capacity, uint32_t flags, void* cuda_stream) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (c->async_open) return fail(c, CDVS_INVALID_ARGUMENT, "asynchronous extractions are pending: call cdvs_wait first");
  if (!c->prop_set) return fail(c, CDVS_INVALID_ARGUMENT, "no cdvs_set_proposal call");
  if (n < 0 || n > kMaxBatch) return fail(c, CDVS_INVALID_ARGUMENT, "n_images must be in 0..4096");
  if (n == 0) return CDVS_OK;
  if (!images || !sizes || !logits_out || capacity < 0) return fail(c, CDVS_INVALID_ARGUMENT, "NULL argument");
  for (int i = 0; i < n; ++i) {
    if (!images[i]) return fail(c, CDVS_INVALID_ARGUMENT, "image pointer is NULL");
    if (sizes[i].width < 16 || sizes[i].height < 16 || sizes[i].width > 32768 || sizes[i].height > 32768 ||
        sizes[i].pitch_bytes < sizes[i].width)
      return fail(c, CDVS_UNSUPPORTED_SIZE, "image sizes must be 16..32768 with pitch >= width");
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  if ((e = cudaSetDevice(c->device)) != cudaSuccess) return cuda_fail(c, e, "device");
  std::vector<const uint8_t*> srcs(images, images + n);
  if (!(flags & CDVS_INPUT_DEVICE)) {
    size_t total = 0;
    std::vector<size_t> off(n);
    for (int i = 0; i < n; ++i) {
      off[i] = total;
      total += ((size_t)sizes[i].pitch_bytes * sizes[i].height + 255) & ~(size_t)255;
    }
    if ((e = ensure(c->input, total)) != cudaSuccess) return cuda_fail(c, e, "input staging");
    for (int i = 0; i < n; ++i) {
      uint8_t* dst = static_cast<uint8_t*>(c->input.p) + off[i];
      if ((e = cudaMemcpyAsync(dst, images[i], (size_t)sizes[i].pitch_bytes * sizes[i].height,
                               cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(c, e, "image upload");
      srcs[i] = dst;
    }
  }
  std::vector<PropImage> t;
  int max_th, max_tw;
  const size_t n_logits = prop_table(n, sizes, srcs.data(), t, max_th, max_tw);
  if (n_logits > (size_t)capacity) return fail(c, CDVS_UNSUPPORTED_SIZE, "logits_out too small");
  const bool dev_out = (flags & CDVS_OUTPUT_DEVICE) != 0;
  if ((e = ensure(c->prop_imgs, sizeof(PropImage) * n)) != cudaSuccess ||
      (!dev_out && (e = ensure(c->prop_logits, sizeof(float) * n_logits)) != cudaSuccess) ||
      (e = cudaMemcpyAsync(c->prop_imgs.p, t.data(), sizeof(PropImage) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(c, e, "proposal workspace");
  float* out = dev_out ? logits_out : static_cast<float*>(c->prop_logits.p);
  if ((e = launch_proposal_infer(static_cast<const PropImage*>(c->prop_imgs.p), n, max_th, max_tw,
                                 static_cast<const float*>(c->prop_theta.p), prop_frag(c), out, s)) != cudaSuccess)
    return cuda_fail(c, e, "proposal launch");
  if (!dev_out && ((e = cudaMemcpyAsync(logits_out, out, sizeof(float) * n_logits, cudaMemcpyDeviceToHost, s)) !=
                       cudaSuccess ||
                   (e = cudaStreamSynchronize(s)) != cudaSuccess))
    return cuda_fail(c, e, "logits readback");
  if ((flags & CDVS_INPUT_DEVICE) == 0 && dev_out && (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(c, e, "proposal");
  return CDVS_OK;
}

cdvs_status cdvs_proposal_train_step(cdvs_ctx* c, const uint8_t* images, int32_t n, int32_t width, int32_t height,
                                     int32_t pitch, const float* labels, float* params, float* adam_m, float* adam_v,
                                     float* grad, float* loss, float* logits, int32_t step, float lr, int32_t bf16,
                                     void* cuda_stream) {
  if (!c) return CDVS_INVALID_ARGUMENT;
  if (c->async_open) return fail(c, CDVS_INVALID_ARGUMENT, "asynchronous extractions are pending: call cdvs_wait first");
  if (!images || !params || !grad || n < 1 || width < 16 || height < 16 || pitch < width || (bf16 != 0 && bf16 != 1))
    return fail(c, CDVS_INVALID_ARGUMENT, "bad training arguments");
  if (lr > 0.0f && (!adam_m || !adam_v || step < 1 || !labels))
    return fail(c, CDVS_INVALID_ARGUMENT, "an update needs labels, Adam moments and step >= 1");
  if ((size_t)n * ((height + 15) / 16) * ((width + 15) / 16) > (size_t)1 << 30 || (size_t)n * height * width > (size_t)1 << 31)
    return fail(c, CDVS_UNSUPPORTED_SIZE, "training batch too large");
  cudaError_t e;
  if ((e = cudaSetDevice(c->device)) != cudaSuccess) return cuda_fail(c, e, "device");
  const size_t nf = proposal_train_floats(n, height, width, c->n_sms);
  if ((e = ensure(c->prop_ws, sizeof(float) * nf)) != cudaSuccess) return cuda_fail(c, e, "training workspace");
  PropTrainArgs t;
  t.images = images;
  t.B = n;
  t.H = height;
  t.W = width;
  t.pitch = pitch;
  t.labels = labels;
  t.theta = params;
  t.adam_m = adam_m;
  t.adam_v = adam_v;
  t.grad = grad;
  t.loss = loss;
  t.logits_out = logits;
  t.step = step;
  t.lr = lr;
  t.bf16 = bf16;
  if ((e = run_proposal_train(t, static_cast<float*>(c->prop_ws.p), c->n_sms, static_cast<cudaStream_t>(cuda_stream))) !=
      cudaSuccess)
    return cuda_fail(c, e, "training step");
  return CDVS_OK;
}

int32_t cdvs_profile_read(cdvs_ctx* c, double* ms, int32_t* launches, int32_t max_stages, int32_t reset) {
  if (!c || !ms || !launches || max_stages < 0) return -1;
  if (cudaSetDevice(c->device) != cudaSuccess) return -1;
  for (int i = 0; i < max_stages; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  for (const ProfRec& r : c->recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return -1;
    if (r.stage < max_stages) {
      ms[r.stage] += t;
      launches[r.stage] += r.launches;
    }
  }
  if (reset) {
    for (const ProfRec& r : c->recs) {
      c->pool.push_back(r.a);
      c->pool.push_back(r.b);
    }
    c->recs.clear();
  }
  return CDVS_N_STAGES;
}

}  // extern "C"
