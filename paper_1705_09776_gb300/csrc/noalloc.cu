// noalloc.cu -- cdvs_dedupe_select_noalloc: the cross-octave check and
// selection of one image with every byte of scratch in a fixed, file-scope
// device array, for callers that must not allocate device memory.
//
// The scratch array below is part of the library image: every GPU that loads
// the library holds it until the process exits.  Host code cannot use the
// array's name as a device address, so the address is looked up once per
// device (cudaGetSymbolAddress, with that device current) and handed to the
// kernels.  All calls share the array: calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it.
//
// The selection kernel checks the caller's records itself (an octave the
// image does not have leaves the record out) and resolves any number of ties
// at the N-th response exactly; what it reports goes to the caller's optional
// device status word, so no synchronisation is needed to learn it.
#include <mutex>

#include "cdvs_internal.cuh"

namespace cdvs {
namespace {

constexpr int kNoAllocMax = CDVS_NOALLOC_MAX_CANDIDATES;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  Cand cand[kNoAllocMax];            // the caller's candidates in octave px
  float4 skey[kNoAllocMax];          // cell-sorted compact copies for the cross-octave check
  int order[kNoAllocMax];            // cell-sorted candidate indices
  unsigned char soct[kNoAllocMax];   // cell-sorted octaves
  unsigned char keep[kNoAllocMax];   // cross-octave check result
  Cand sel[kMaxSelect];              // selected points in rank order
  ImgPlan plan;                      // size and octave count of the image
  int cand_count;
  int sel_count;
  int status;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_lock[kMaxDevices];
NoAllocScratch* g_addr[kMaxDevices];

// Caller records -> octave-px candidates; clears the counters and status.  A
// record whose octave is outside 0 .. n_oct - 1 keeps octave -1, which the
// selection kernel leaves out (and reports).
__global__ void noalloc_in_kernel(NoAllocScratch* s, const cdvs_keypoint* cand, int n, int W, int H, int n_oct) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    s->plan.W = W;
    s->plan.H = H;
    s->plan.n_oct = n_oct;
    s->cand_count = n;
    s->sel_count = 0;
    s->status = 0;
  }
  if (i < n) {
    const cdvs_keypoint k = cand[i];
    const bool ok = k.octave >= 0 && k.octave < n_oct;
    const float inv = ok ? 1.0f / (float)(1 << k.octave) : 0.0f;
    Cand c;
    c.xo = k.x * inv;
    c.yo = k.y * inv;
    c.so = k.sigma * inv;
    c.resp = k.response;
    c.pss = k.p_ss;
    c.ratio = k.ratio;
    c.octave = ok ? k.octave : -1;
    c.type = k.type;
    c.spare = i;
    s->cand[i] = c;
  }
}

// Selected points -> caller records (image 0, parent_id = index in the input),
// the count, and the call's status code when the caller asked for it.
__global__ void noalloc_out_kernel(const NoAllocScratch* s, cdvs_keypoint* out, int* out_count, int* out_status) {
  const int n = s->sel_count;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *out_count = n;
    if (out_status) {
      const int st = s->status;
      *out_status = (st & kStatusBadInput)          ? CDVS_INVALID_ARGUMENT
                    : (st & kStatusSelectOverflow) ? CDVS_CAPACITY_TRUNCATED
                                                   : CDVS_OK;
    }
  }
  if (i < n) {
    const Cand& q = s->sel[i];
    const float sc = (float)(1 << q.octave);
    cdvs_keypoint k;
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
    k.image = 0;
    k.parent_id = q.spare;
    out[i] = k;
  }
}

// Device address of the scratch array on the current device.  Only a
// successful lookup is kept: a failed one (say, made during a stream
// capture) is tried again on the next call.
cudaError_t scratch_address(int device, NoAllocScratch** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_lock[device]);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    g_addr[device] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace
}  // namespace cdvs

using namespace cdvs;

extern "C" cdvs_status cdvs_dedupe_select_noalloc(const cdvs_keypoint* cand, int32_t n_cand, int32_t width,
                                                  int32_t height, const cdvs_params* params,
                                                  cdvs_keypoint* sel_out, int32_t* sel_count, int32_t* dev_status,
                                                  void* cuda_stream) {
  if (!params || !sel_out || !sel_count || n_cand < 0 || (n_cand > 0 && !cand)) return CDVS_INVALID_ARGUMENT;
  if (n_cand > kNoAllocMax) return CDVS_UNSUPPORTED_SIZE;
  if (width < 16 || height < 16 || width > 32768 || height > 32768) return CDVS_UNSUPPORTED_SIZE;
  if (params->max_keypoints < 1 || params->max_keypoints > kMaxSelect || !(params->dedupe_dlog2 >= 0.0f) ||
      params->num_octaves < 1 || params->num_octaves > kMaxOctaves)
    return CDVS_INVALID_ARGUMENT;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return CDVS_CUDA_ERROR;
  NoAllocScratch* s = nullptr;
  if (scratch_address(device, &s) != cudaSuccess || !s) return CDVS_CUDA_ERROR;
  int n_oct = 0;
  for (int w = width, h = height; n_oct < params->num_octaves && w >= 3 && h >= 3; ++n_oct) {
    w = (w + 1) / 2;
    h = (h + 1) / 2;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int n_in = n_cand > 0 ? n_cand : 1;
  noalloc_in_kernel<<<(n_in + 255) / 256, 256, 0, st>>>(s, cand, n_cand, width, height, n_oct);
  if (cudaGetLastError() != cudaSuccess) return CDVS_CUDA_ERROR;
  SelectArgs a;
  a.plans = &s->plan;
  a.cands = s->cand;
  a.cand_count = &s->cand_count;
  a.cand_cap = kNoAllocMax;
  a.order = s->order;
  a.keep = s->keep;
  a.skey = s->skey;
  a.soct = s->soct;
  a.sel = s->sel;
  a.sel_count = &s->sel_count;
  a.N = params->max_keypoints;
  a.dlog2 = params->dedupe_dlog2;
  a.status = &s->status;
  if (launch_select(a, 1, st) != cudaSuccess) return CDVS_CUDA_ERROR;
  noalloc_out_kernel<<<(params->max_keypoints + 255) / 256, 256, 0, st>>>(s, sel_out, sel_count, dev_status);
  if (cudaGetLastError() != cudaSuccess) return CDVS_CUDA_ERROR;
  return CDVS_OK;
}
