// cdvs_internal.cuh -- device-side data layout and kernel interfaces of the
// GB300 CDVS front end.  Shared by the .cu files of this library only.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/cdvs.h"

namespace cdvs {

// ---------------------------------------------------------------- limits
constexpr int kMaxOctaves = 12;
constexpr int kScales = 4;       // K: levels per octave fitted by the cubic (Eq. 2-3)
constexpr int kMaxRadius = 24;   // largest Gaussian radius a level filter may have
constexpr int kMaxOri = 8;       // orientation copies per point
constexpr int kMaxSelect = 2048; // N limit of the selection step
constexpr int kSelectList = 4096;  // most entries sorted by the selection step (N + ties)
constexpr int kMaxCells = 8192;  // spatial hash cells of the cross-octave check
constexpr int kMaxBatch = 4096;  // images per call (the detection tile list lives in shared memory)

// detection tile (output pixels per CTA) and CTA size
constexpr int kTX = 128;
constexpr int kTY = 32;
constexpr int kDetThreads = 512;
constexpr int kHalo = 2;         // 1 px for the Laplacian + 1 px for the 8-neighbour test

// status word bits (device), OR-ed by kernels
constexpr int kStatusCandOverflow = 1;
constexpr int kStatusSelectOverflow = 2;
constexpr int kStatusOutTruncated = 4;
constexpr int kStatusTimeout = 8;        // a bounded device-side wait gave up
constexpr int kStatusBadInput = 16;      // a caller record was out of range and was left out

// ---------------------------------------------------------------- plans
// Level (o, k) of an image is stored at level_base + oct[o].level_off +
// k * oct[o].lpitch * oct[o].H elements (FP32 or FP16), rows lpitch apart.
// An octave's levels are stored either in the image's orientation or
// transposed (a stored row is an image column), whichever covers the octave
// with fewer detection tiles; W, H, lpitch and the tiles are those of the
// stored frame.
struct OctPlan {
  int W, H;
  int lpitch;          // elements per stored row (multiple of 8)
  int tiles_x, tiles_y;
  int tr;              // 1: stored transposed
  long long level_off; // element offset of level (o, 0) in the level arena
};

struct ImgPlan {
  const uint8_t* src;  // device pointer to the 8-bit image
  int W, H, pitch;     // pitch in bytes
  int n_oct;
  OctPlan oct[kMaxOctaves];
};

// One candidate / selected point, octave px.  32 bytes.
struct Cand {
  float xo, yo, so;    // position and scale in octave px
  float resp;          // refined response p-hat
  float pss;           // d2p/dsigma2 at sigma*
  float ratio;         // Hessian tr^2/det
  short octave, type;  // octave; +1 max / -1 min
  int spare;
};

// ---------------------------------------------------------------- K1 args
struct DetectArgs {
  const ImgPlan* plans;
  const int* tile_prefix;  // n_images + 1 entries: first tile of each image, minus tile_base
  int tile_base;
  int n_images;
  int octave;
  void* levels;            // level arena (float or __half)
  Cand* cands;             // n_images x cand_cap
  int* cand_count;         // per image
  int cand_cap;
  int* status;
  int radius[kScales];
  float2 taps[kScales][kMaxRadius + 1];  // one side of each symmetric level filter, each tap as a pair
                                         // {g, g} (the operand of a packed FP32 multiply-add)
  float s2[kScales];                     // s_k^2: LoG scale normalisation
  float B[4][kScales];                   // cubic fit in t = sigma - tc: a_i = sum_k B[i][k] L_k
  float tc;                              // centre of the fitting variable
  float t_lo, t_hi;                      // admissible t range (s_0 - tc, s_{K-1} - tc)
  float T;                               // contrast threshold
  float edge_lim;                        // (r+1)^2 / r
  float offset_max;
  int write_level0;                      // 1 at octave 0 (level 0 is filtered, not the base)
  const uint8_t* tile_mode;              // per tile of the batch (index tile_base + b), or null: all detect
  const uint16_t* block_mask;            // per tile: its 8 x 2 blocks of 16 x 16 px (bit 8 row + col) where
                                         // detection keeps survivors, or null: all
};

// What K1 does with a tile when a block proposal masks the first octave
constexpr uint8_t kModeLevel3 = 0;  // level 3 and the next octave's base only
constexpr uint8_t kModeLevels = 1;  // every level stored (description may read them), no detection
constexpr uint8_t kModeDetect = 2;  // the whole of Alg. 1 on the tile

// ---------------------------------------------------------------- K3/K10 args
struct SelectArgs {
  const ImgPlan* plans;
  const Cand* cands;
  const int* cand_count;
  int cand_cap;
  int* order;              // scratch n_images x cand_cap: candidate index at each cell-sorted position
  unsigned char* keep;     // scratch n_images x cand_cap
  float4* skey;            // scratch n_images x cand_cap: cell-sorted (x, y, sigma in image px, |response|)
  unsigned char* soct;     // scratch n_images x cand_cap: cell-sorted octaves
  Cand* sel;               // n_images x N
  int* sel_count;
  int N;
  float dlog2;
  int* status;
  int list_cap;            // entries of the tie list sorted per image (set by launch_select)
};

// ---------------------------------------------------------------- K5/K6 args
struct DescribeArgs {
  const ImgPlan* plans;
  const void* levels;
  const Cand* sel;         // n_images x N
  const int* sel_count;
  int N;
  int n_images;
  float* ori_theta;        // n_images x N x kMaxOri
  int* ori_count;          // n_images x N
  int* rec_off;            // packing scratch: per-slot and per-image record offsets
  int* rec_total;          // number of records written
  int* kp_count;           // per image records written
  int kp_capacity;
  cdvs_keypoint* kp_out;
  float* desc_out;
  int* status;
  float sigma0;
  int upright;
  int max_ori;
  float ori_radius, ori_ratio, ori_wsig;
  float desc_radius, cell_side, desc_wsig;
  int patch_side;               // staged patch side (pixels) per point
  cdvs_keypoint* stage_kp;      // n_images x N x max_ori staging slots
  float* stage_desc;            // n_images x N x max_ori x 128
  // the launch's image group [img_begin, img_end); its counters (zeroed
  // before the call): slot claims of the description, CTAs done in the
  // scan; the group's first record (base_in) and the next group's (base_out)
  int img_begin, img_end;
  unsigned* claim;
  unsigned* scan_done;
  const int* base_in;
  int* base_out;
  int last_group;               // 1: the scan also writes the batch total and the truncation bit
};

// Host-side launch set-up of one kernel, per device: the largest dynamic
// shared memory it was allowed so far and its occupancy at the last size
// asked.  cudaFuncSetAttribute and the occupancy query cost microseconds of
// host time each, which a call of one small image would pay at every launch;
// here they run once per kernel, device and size.
struct LaunchCache {
  static constexpr int kDevices = 16;
  std::mutex m;
  int smem_set[kDevices] = {};
  int occ_for[kDevices] = {};  // shared memory + 1 of the cached occupancy (0: none)
  int occ[kDevices] = {};
};

// Allows `smem` bytes of dynamic shared memory for `func` on the current
// device and, when per_sm is given, returns how many CTAs of `threads`
// threads fit on an SM.
template <typename F>
cudaError_t prepare_launch(F* func, LaunchCache& c, int smem, int threads, int* per_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= LaunchCache::kDevices) {
    if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    return per_sm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, func, threads, smem) : cudaSuccess;
  }
  std::lock_guard<std::mutex> lock(c.m);
  if (smem > c.smem_set[dev]) {
    if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    c.smem_set[dev] = smem;
  }
  if (per_sm) {
    if (c.occ_for[dev] != smem + 1) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ[dev], func, threads, smem)) != cudaSuccess)
        return e;
      c.occ_for[dev] = smem + 1;
    }
    *per_sm = c.occ[dev];
  }
  return cudaSuccess;
}

// launchers (defined in the .cu files)
size_t detect_smem_bytes(int max_radius);
// K1 variants (work shapes of the same arithmetic; every variant gives the
// same levels and candidates bit for bit): 0 and 1 tile 128 x 32 with one
// 512-thread CTA per SM, 2 and 3 tile 128 x 16 with two 256-thread CTAs per
// SM; they differ in the rows per thread of the y pass.
constexpr int kDetectVariants = 4;
int detect_variant_rows(int variant);          // output rows of the variant's tile
const char* detect_variant_name(int variant);
cudaError_t launch_detect(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, int variant,
                          cudaStream_t s);
cudaError_t launch_detect_a(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, cudaStream_t s);
cudaError_t launch_detect_b(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, cudaStream_t s);
cudaError_t launch_detect_c(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, cudaStream_t s);
cudaError_t launch_detect_d(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms, cudaStream_t s);
cudaError_t launch_detect_masked(const DetectArgs& a, int n_tiles, int max_radius, int storage, int n_sms,
                                 cudaStream_t s);
cudaError_t launch_select(const SelectArgs& a, int n_images, cudaStream_t s);
size_t describe_smem_bytes(int patch_side);
cudaError_t launch_describe(const DescribeArgs& a, int storage, int n_sms, cudaStream_t s);
constexpr int kMaxOutGroups = 4;  // image groups the description and packing kernels can be launched on
cudaError_t launch_pack(const DescribeArgs& a, cudaStream_t s);
cudaError_t launch_copy(const DescribeArgs& a, int n_sms, cudaStream_t s);
// One stored level (W x H in the stored frame, transposed when tr) -> FP32
// in the image's orientation, rows of the image width.
cudaError_t launch_levels_to_f32(const void* levels, int storage, int W, int H, int tr, long long off, int lpitch,
                                 float* out, cudaStream_t s);

// ---------------------------------------------------------------- proposal
constexpr int kPropParams = 4817;  // W1 144, b1 16, W2 2304, b2 16, W3 2304, b3 16, Wh 16, bh 1

struct PropImage {
  const uint8_t* src;
  int W, H, pitch;
  int H1, W1, H2, W2;  // conv1 and conv2/conv3 output sizes
  int Th, Tw;          // 16x16 blocks
  int logit_off;       // first logit of the image
};

struct PropTrainArgs {
  const uint8_t* images;  // B images of H x W, row pitch `pitch`, back to back
  int B, H, W, pitch;
  const float* labels;    // B x Th x Tw in {0, 1}, or null: forward only
  float* theta;           // kPropParams FP32 (updated when lr > 0)
  float* adam_m;
  float* adam_v;
  float* grad;            // kPropParams
  float* loss;            // mean BCE (1 float), may be null
  float* logits_out;      // B x Th x Tw, may be null
  int step;               // Adam step (from 1)
  float lr;               // 0: no update
  int bf16;               // 1: BF16 weights and A1/A2, as in inference
};

size_t proposal_infer_smem();
constexpr int kPropFragWords = 2 * 9 * 2 * 32 * 2;  // conv2/conv3 B fragments (uint32)
void pack_proposal_fragments(const float* theta, uint32_t* frag);
cudaError_t launch_proposal_infer(const PropImage* d_imgs, int n_images, int max_th, int max_tw, const float* theta,
                                  const uint32_t* frag, float* logits, cudaStream_t s);
cudaError_t launch_tile_mode(const PropImage* d_imgs, const ImgPlan* plans, const int* tile_prefix, int n_images,
                             int max_blocks, int max_tiles, const float* logits, float zt, int dil, int ny, int nx,
                             uint8_t* mode, uint16_t* block_mask, uint8_t* near, uint8_t* det, cudaStream_t s);
size_t proposal_train_floats(int B, int H, int W, int n_sms);
cudaError_t run_proposal_train(const PropTrainArgs& t, float* ws, int n_sms, cudaStream_t s);

// ---------------------------------------------------------------- S0 resize
struct ResizeJob {
  const uint8_t* src;
  int W, H, pitch;
  uint8_t* dst;
  int W2, H2, pitch2;
};
cudaError_t launch_resize(const ResizeJob* d_jobs, int n_jobs, int max_rows, cudaStream_t s);

// ---------------------------------------------------------------- SCFV
constexpr int kScfvComp = 512, kScfvDim = 32;
// the device model, derived on the host: P transposed [128][32], the PCA
// mean, mu [512][32], 1/s [512][32], log w_i - 1/2 sum_k log(2 pi v_ik),
// 1/sqrt(w_i), 1/sqrt(2 w_i); then the matrix form of the log-likelihood
// (Eq. 10), W [64][512] with rows k < 32 = -1/(2 v_ik) (the y_k^2 terms) and
// rows 32 + k = mu_ik / v_ik (the y_k terms), as the tcgen05 B operand: per
// component i, column i of W times a power of two e_i (largest |entry| at most
// 2^14), split into FP16 hi and lo halves, each half [512][64] in the
// no-swizzle K-major core-matrix order (kScfvTcBIndex, in halves); the
// constant c_i = log w_i - 1/2 sum_k log(2 pi v_ik) - 1/2 sum_k mu_ik^2 / v_ik;
// 1 / e_i; and P transposed as FP16 hi / lo B fragments of mma.sync
// m16n8k16 (kScfvPfIndex, half2 words).
constexpr int kScfvOffPcaT = 0, kScfvOffMean = 4096, kScfvOffMu = 4224, kScfvOffIsd = 20608, kScfvOffLw = 36992,
              kScfvOffNmu = 37504, kScfvOffNsig = 38016, kScfvOffW = 38528, kScfvOffC = 71296,
              kScfvOffInvE = 71808, kScfvOffPf = 72320, kScfvModelFloats = 76416;
constexpr int kScfvWHalfWords = 16384;  // one FP16 half of the B operand, in 32-bit words
// Position (in halves) of B element (component i, row k of W) in one half:
// 8 x 8 core matrices of 128 contiguous bytes, adjacent along k at 128
// bytes, along i at 1024 bytes.
inline int kScfvTcBIndex(int i, int k) { return (i / 8) * 512 + (k / 8) * 64 + (i % 8) * 8 + (k % 8); }
// Position (in half2 words) of the projection fragment holding P^T rows
// (input dimensions) 2t + 8q, 2t + 8q + 1 of k-step s and output column
// 8 j8 + g (lane 4 g + t); the lo halves follow 2048 words later.
inline int kScfvPfIndex(int s, int j8, int lane, int q) { return ((s * 4 + j8) * 32 + lane) * 2 + q; }
// The measured packed-FP32 FMA rate of the current device (probe.cu).
cudaError_t probe_ffma2(int n_sms, double* tflops);
// The bytes of the operands the posterior kernel writes for the gradient
// products (32-record chunks of the batch).
size_t scfv_ops_bytes(int n_rec);
cudaError_t launch_scfv(const float* desc, int n_rec, const int* rec_off, int n_images, const float* model,
                        int n_select, void* ops, float* g_mu, float* g_sig, float* delta, int* order,
                        uint32_t* bits, int* status, int skip_products, int n_sms, cudaStream_t s);

}  // namespace cdvs
