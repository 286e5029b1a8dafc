/*
 * cdvs.h -- C ABI of the GB300 (sm_103a) CDVS front end: interest point
 * detection and local feature description of the MPEG-CDVS encoder as
 * moved to the GPU in "Fast MPEG-CDVS Encoder with GPU-CPU Hybrid Computing"
 * (arXiv 1705.09776), Sec. IV-A (Alg. 1) and Sec. IV-B (Alg. 2), plus the
 * feature selection of Sec. III-B (Eq. 5) and the host-side descriptor
 * transform and ternary quantisation of Sec. III-C.
 *
 * Conventions
 *   - Images are 8-bit grey, row-major, `pitch_bytes` between rows.
 *   - Coordinates: pixel centres at integer positions, origin at the centre
 *     of the top-left pixel, x to the right, y down.  "Image px" are input
 *     pixels; pixel i of octave o sits on image pixel 2^o * i ("octave px").
 *   - Angles are radians in [0, 2 pi), measured from +x towards +y.
 *   - Every call is asynchronous on `cuda_stream` (a cudaStream_t, NULL for
 *     the legacy default stream) unless it reads results back to host memory,
 *     in which case it returns after they are in place.
 *   - No exception crosses this boundary.  Every call returns a cdvs_status;
 *     on anything but CDVS_OK / CDVS_CAPACITY_TRUNCATED the outputs are
 *     unspecified and cdvs_last_error() describes the failure.
 *   - Ownership: the caller owns every input and output buffer (host or
 *     device, as `flags` says) and the library never frees them.  The
 *     context owns its device workspace and grows it on demand.  Calls on one
 *     context must not overlap (one context per host thread); distinct
 *     contexts are independent.
 */
#ifndef CDVS_H
#define CDVS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CDVS_OK = 0,
    CDVS_INVALID_ARGUMENT = 1,   /* null pointer, bad count, parameter out of range */
    CDVS_UNSUPPORTED_SIZE = 2,   /* image side < 16 px or > 32768 px */
    CDVS_OUT_OF_MEMORY = 3,      /* device or pinned host allocation failed */
    CDVS_CAPACITY_TRUNCATED = 4, /* an output or internal queue was full; results truncated */
    CDVS_DEVICE_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    CDVS_CUDA_ERROR = 6          /* a CUDA runtime call failed (message in cdvs_last_error) */
} cdvs_status;

/* flags */
#define CDVS_INPUT_DEVICE 0x1u   /* image pointers (and point lists) are device memory */
#define CDVS_OUTPUT_DEVICE 0x2u  /* output buffers are device memory */
#define CDVS_ASYNC 0x4u          /* cdvs_extract only: see cdvs_wait */

/* Level storage types (cdvs_params.storage). */
#define CDVS_STORAGE_FP32 0
#define CDVS_STORAGE_FP16 1

typedef struct cdvs_ctx cdvs_ctx;

/* Parameters of the method.  cdvs_params_default() fills the values below;
 * the paper fixes 3.96, 0.8, 6 and 3 (Sec. IV-B) and about 300 features
 * (Sec. III-B); the rest are this library's readings where the paper is
 * silent. */
typedef struct {
    int32_t num_octaves;       /* octaves processed at most (4); an octave needs both sides >= 3 */
    int32_t scales_per_octave; /* K LoG scales per octave fitted by the cubic of Eq. 2 (4; only 4) */
    float sigma0;              /* scale of level 0 of each octave, octave px (1.6) */
    float sigma_in;            /* blur assumed present in the input (0.5) */
    float contrast_T;          /* threshold on |p| at sigma* and after refinement (4.0, grey levels) */
    float edge_r;              /* Hessian edge ratio r: reject tr^2/det >= (r+1)^2/r (10) */
    float offset_max;          /* reject refined offsets above this, octave px (0.5) */
    float ori_radius;          /* orientation disc radius in sigma (3.96) */
    float ori_peak_ratio;      /* keep histogram peaks above this fraction of the max (0.8) */
    float ori_weight_sigma;    /* orientation Gaussian weight std in sigma (1.5) */
    float desc_radius;         /* description disc radius in sigma (6.0) */
    float cell_side;           /* descriptor cell side in sigma (3.0) */
    float desc_weight_sigma;   /* descriptor Gaussian weight std in cells (2.0) */
    float dedupe_dlog2;        /* cross-octave duplicate window on |log2 sigma ratio| (1/3) */
    int32_t max_keypoints;     /* N points kept by selection, 1..2048 (300) */
    int32_t max_orientations;  /* orientation copies per point, 1..8 (4) */
    int32_t upright;           /* 1: theta = 0 and no orientation stage (0) */
    int32_t storage;           /* CDVS_STORAGE_FP32 or CDVS_STORAGE_FP16 level storage (FP32) */
    int32_t use_proposal;      /* 1: the learned block proposal masks first-octave detection in
                                  cdvs_extract and cdvs_candidates (0; needs cdvs_set_proposal) */
    float proposal_threshold;  /* a 16x16 block is proposed when its probability exceeds this (0.5) */
    int32_t max_side;          /* S0: an image whose larger side exceeds this is first resized by area
                                  averaging to that side (0 = never; 640 for uneven batches); its
                                  records are then in the resized image's pixels */
} cdvs_params;

typedef struct {
    int32_t width, height;  /* pixels */
    int32_t pitch_bytes;    /* bytes between rows, >= width */
} cdvs_image_desc;

/* One interest point, or one (point, orientation) output record.  44 bytes. */
typedef struct {
    float x, y, sigma;      /* image px */
    float theta;            /* orientation, radians (0 for candidates and in upright mode) */
    float response;         /* refined scale-normalised LoG response p-hat (Alg. 1 stage B) */
    float p_ss;             /* d2p/dsigma2 at sigma*, octave px units (Eq. 5 input) */
    float ratio;            /* Hessian tr^2/det (Eq. 5 input) */
    int16_t octave;         /* octave o */
    int16_t scale_idx;      /* Gaussian level used for description */
    int16_t type;           /* +1 maximum, -1 minimum */
    int16_t reserved;
    int32_t image;          /* index of the image in the call */
    int32_t parent_id;      /* rank of the selected point (descriptor records) */
} cdvs_keypoint;

/* Fills *p with the defaults listed above. */
void cdvs_params_default(cdvs_params *p);

/* Creates a context on CUDA device `device`.  `workspace_bytes_hint` (may be
 * 0) pre-allocates that much device workspace.  Returns CDVS_OK and *out, or
 * an error (then *out is NULL). */
cdvs_status cdvs_create(cdvs_ctx **out, int device, size_t workspace_bytes_hint);

/* Destroys a context and frees its workspace.  NULL is a no-op. */
void cdvs_destroy(cdvs_ctx *ctx);

/* Message of the last failed call on ctx ("" if none).  Valid until the next
 * call on ctx. */
const char *cdvs_last_error(const cdvs_ctx *ctx);

/*
 * cdvs_extract -- the whole front end on a batch: Gaussian scale space
 * (Eq. 1, Alg. 1 stage A), LoG and ALP cubic-in-scale extremum detection
 * (Eq. 2-3), refinement (Alg. 1 stage B), cross-octave duplicate removal
 * (Alg. 1 stage C), selection of the N best points (Eq. 5, |p-hat| standing in
 * for the normative relevance tables), dominant orientations (Alg. 2 stage A)
 * and 128-D descriptors (Alg. 2 stage B).
 *
 *   n_images       0 .. 4096 images in one call
 *   images[i]      pointer to image i (host, or device with CDVS_INPUT_DEVICE)
 *   sizes[i]       its width, height and pitch (host memory)
 *   kp_out         kp_capacity records, packed over the batch: the records of
 *                  image i follow those of image i-1, each image's in rank order
 *                  then orientation order (peak value descending)
 *   desc_out       kp_capacity * 128 floats (16-byte aligned when on the
 *                  device), descriptor j belongs to record j:
 *                  cells row-major (y, x) in the rotated frame, 8 orientation
 *                  bins fastest; unit L2 norm
 *   kp_count[i]    records written for image i (host, or device with
 *                  CDVS_OUTPUT_DEVICE)
 *   flags          CDVS_INPUT_DEVICE, CDVS_OUTPUT_DEVICE, CDVS_ASYNC (return once
 *                  the batch is enqueued; see cdvs_wait)
 * Returns CDVS_CAPACITY_TRUNCATED if kp_capacity was too small (records are
 * dropped from the end of the batch) or an image had more candidates than the
 * internal queue holds.
 */
cdvs_status cdvs_extract(cdvs_ctx *ctx, int32_t n_images, const uint8_t *const *images,
                         const cdvs_image_desc *sizes, const cdvs_params *params,
                         cdvs_keypoint *kp_out, float *desc_out, int32_t kp_capacity,
                         int32_t *kp_count, uint32_t flags, void *cuda_stream);

/*
 * cdvs_wait -- completes asynchronous extractions.  A cdvs_extract call with
 * CDVS_ASYNC returns as soon as its batch is enqueued, with CDVS_OK or an
 * argument error, so the host prepares and enqueues the next batch while the
 * GPU works on this one.
 *   Device outputs are complete when `cuda_stream` reaches the call.
 *   Host outputs (kp_out, desc_out, kp_count) are copied out once the call's
 *   record total is known: the copies are enqueued by the next asynchronous
 *   call (which first waits until this call's records are packed) or by
 *   cdvs_wait, on a copy stream of the context, so they overlap the next
 *   batch.  Host images are copied in by the call itself.  Host buffers of
 *   both directions must stay valid and unchanged until cdvs_wait returns;
 *   page-locked memory keeps the copies asynchronous.
 * cdvs_wait enqueues what is pending, synchronises `cuda_stream` (the stream
 * of those calls) and the copies, and returns what the calls since the
 * previous cdvs_wait reported together: CDVS_CAPACITY_TRUNCATED if any of
 * them truncated, else CDVS_OK.  Asynchronous calls on one context must use
 * one stream, and no other call that uses the context's workspace is
 * accepted until cdvs_wait (INVALID_ARGUMENT).  The context alternates two
 * staging sets (page-locked tables, device copies of host images and of
 * host-bound records), so enqueueing a call waits at most for the call two
 * before it.
 */
cdvs_status cdvs_wait(cdvs_ctx *ctx, void *cuda_stream);

/*
 * cdvs_candidates -- Alg. 1 stages A and B only: every refined candidate of
 * every octave, before the cross-octave check and selection, packed over the
 * batch (per image in no particular order).  theta = 0, parent_id = -1.
 */
cdvs_status cdvs_candidates(cdvs_ctx *ctx, int32_t n_images, const uint8_t *const *images,
                            const cdvs_image_desc *sizes, const cdvs_params *params,
                            cdvs_keypoint *cand_out, int32_t cand_capacity, int32_t *cand_count,
                            uint32_t flags, void *cuda_stream);

/*
 * cdvs_dedupe_select -- Alg. 1 stage C and the selection of Eq. 5 on given
 * candidates: cand[i * cand_stride + j], j < cand_count[i], are image i's
 * candidates (fields x, y, sigma, response, octave used; octave px positions
 * are x / 2^octave; an octave the image does not have is INVALID_ARGUMENT).
 * Writes the selected points in rank order, packed over the batch, with
 * parent_id = the candidate's index j.  Any number of candidates tying at the
 * N-th response is resolved by the total order (|response| desc, y, x,
 * sigma, octave asc), whatever their order in cand.  Host buffers only.
 */
cdvs_status cdvs_dedupe_select(cdvs_ctx *ctx, int32_t n_images, const cdvs_image_desc *sizes,
                               const cdvs_keypoint *cand, const int32_t *cand_count,
                               int32_t cand_stride, const cdvs_params *params,
                               cdvs_keypoint *sel_out, int32_t sel_capacity, int32_t *sel_count,
                               uint32_t flags, void *cuda_stream);

/*
 * cdvs_describe -- Alg. 2 on given points: builds each image's scale space,
 * then orientations and descriptors of pts[i * pts_stride + j], j < n_pts[i]
 * (fields x, y, sigma, octave used).  Output as cdvs_extract; parent_id is j.
 */
cdvs_status cdvs_describe(cdvs_ctx *ctx, int32_t n_images, const uint8_t *const *images,
                          const cdvs_image_desc *sizes, const cdvs_params *params,
                          const cdvs_keypoint *pts, const int32_t *n_pts, int32_t pts_stride,
                          cdvs_keypoint *kp_out, float *desc_out, int32_t kp_capacity,
                          int32_t *kp_count, uint32_t flags, void *cuda_stream);

/*
 * cdvs_scale_space -- the Gaussian levels G_{o,k} of one image (Eq. 1,
 * Alg. 1 stage A, octave downsampling of Alg. 1), as FP32 MINUS 128 (the
 * library filters the input shifted by -128, which keeps FP32 rounding small;
 * the shift cancels in every difference).  Levels are written octave-major,
 * then level, then row-major without padding: level (o, k) has W_o x H_o
 * values, W_{o+1} = ceil(W_o / 2).  `capacity` is in floats; `*n_octaves`
 * gets the number of octaves.  Host buffer unless CDVS_OUTPUT_DEVICE.
 */
cdvs_status cdvs_scale_space(cdvs_ctx *ctx, const uint8_t *image, const cdvs_image_desc *size,
                             const cdvs_params *params, float *levels_out, size_t capacity,
                             int32_t *n_octaves, uint32_t flags, void *cuda_stream);

/*
 * Measurement hooks (no counterpart in the paper; they only time it).
 * cdvs_profile(ctx, 1) makes every later call on ctx record CUDA events on
 * its stream around each kernel stage; cdvs_profile_read() waits for the
 * recorded events, adds each stage's elapsed device time (ms) and launch
 * count to ms[s] / launches[s] for stage s in
 *   0 detect (one launch per octave), 1 dedupe + select, 2 orientation and
 *   descriptors, 3 record offsets, 4 record packing, 5 the octave-0 detect
 *   launch alone (part of stage 0), 6 the block proposal network and the
 *   tile modes (params->use_proposal = 1 only),
 * and clears the record when `reset` is nonzero.  Returns the number of
 * stages (7) or -1 on error.
 */
#define CDVS_N_STAGES 7
cdvs_status cdvs_profile(cdvs_ctx *ctx, int32_t enable);
int32_t cdvs_profile_read(cdvs_ctx *ctx, double *ms, int32_t *launches, int32_t max_stages,
                          int32_t reset);

/*
 * cdvs_rank_host -- the selection order of Eq. 5 on the host (pure CPU,
 * deterministic): indices of the n points sorted by |response| descending,
 * then y, x, sigma, octave ascending; at most max_keypoints written to
 * `order`.  Returns the number written.  This is the same total order the
 * device selection uses, for re-ranking records on the host.
 */
int32_t cdvs_rank_host(const cdvs_keypoint *pts, int32_t n, int32_t max_keypoints,
                       int32_t *order);

/*
 * cdvs_transform_ternary -- Sec. III-C on the host (pure CPU, FP64
 * arithmetic): each of the 16 cell histograms h0..h7 of a descriptor goes
 * through one of two order-8 add/subtract/shift transforms (set A for cells
 * with cx + cy even, set B otherwise), and each transformed value v_j becomes
 * -1 if v_j < t_lo[j], +1 if v_j > t_hi[j], else 0.  desc: n x 128 floats;
 * t_lo, t_hi: 128 thresholds each; out: n x 128 int8.  v_out (may be NULL)
 * receives the transformed values as n x 128 doubles.
 */
cdvs_status cdvs_transform_ternary(const float *desc, int32_t n, const double *t_lo,
                                   const double *t_hi, int8_t *out, double *v_out);

/*
 * cdvs_dedupe_select_noalloc -- the cross-octave check and selection of
 * cdvs_dedupe_select for ONE image, without allocating any memory.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc, for example code that runs with a fixed device-memory
 * budget reserved at start-up, or code that must not add allocations while
 * other threads capture CUDA graphs (an allocation there can break or
 * serialise the capture).
 *
 * Its scratch (converted candidates, cell order, check flags, selected
 * points; about 930 KB) is a fixed array inside the library, so every GPU
 * that loads the library keeps that much device memory until the process
 * exits.  The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress); make that first call before any stream capture (a
 * lookup that fails is not remembered: the next call tries again).
 * All calls share the one array and it keeps the last call's contents: calls
 * whose GPU work overlaps (other streams, other host threads) race and give
 * wrong results -- serialise them.
 *
 *   cand       n_cand candidate records in DEVICE memory (fields x, y, sigma,
 *              response, p_ss, ratio, octave, type used); octave is one of
 *              the image's octaves (0 .. octaves of width x height - 1)
 *   n_cand     0 .. CDVS_NOALLOC_MAX_CANDIDATES; more -> CDVS_UNSUPPORTED_SIZE
 *              (nothing is launched)
 *   width, height  image size (16..32768) the candidates come from
 *   sel_out    DEVICE memory for params->max_keypoints records, written in
 *              rank order with image = 0 and parent_id = index in cand
 *   sel_count  DEVICE int, receives the number of selected points
 *   dev_status DEVICE int or NULL; receives, when the work has run, CDVS_OK,
 *              CDVS_INVALID_ARGUMENT (a record's octave was not one of the
 *              image's octaves: that record was left out, the others
 *              selected), or CDVS_CAPACITY_TRUNCATED (more than 4096
 *              records identical in response, position, scale and octave
 *              tie at the N-th rank; not met with real candidates)
 * Runs asynchronously on cuda_stream on the current device.  The return
 * value covers the arguments and the launches only (CDVS_OK once the work is
 * queued); what the GPU finds goes to dev_status, so reading it needs no
 * synchronisation inside this call.
 */
#define CDVS_NOALLOC_MAX_CANDIDATES 16384
cdvs_status cdvs_dedupe_select_noalloc(const cdvs_keypoint *cand, int32_t n_cand, int32_t width,
                                       int32_t height, const cdvs_params *params,
                                       cdvs_keypoint *sel_out, int32_t *sel_count,
                                       int32_t *dev_status, void *cuda_stream);

/* enable = 1: calls of cdvs_extract with both CDVS_INPUT_DEVICE and
 * CDVS_OUTPUT_DEVICE (and profiling off) capture their device work -- input
 * tables, every kernel of the batch, the status read -- into a CUDA graph,
 * update the context's executable graph with it in place (instantiating it
 * again when the work changed shape) and launch that.  Results are
 * unchanged.  0 turns it off and frees the graph. */
cdvs_status cdvs_set_graph(cdvs_ctx *ctx, int32_t enable);

/* S0 alone: each image whose larger side exceeds max_side is resized by area
 * averaging (see cdvs_params.max_side), the others are copied.  Output image
 * i is written to out (row pitch = its width) after images 0..i-1, and its
 * size to out_sizes[i]; capacity is the size of out in bytes
 * (UNSUPPORTED_SIZE when too small).  flags: CDVS_INPUT_DEVICE,
 * CDVS_OUTPUT_DEVICE (out in device memory; out_sizes is always host
 * memory).  Synchronous unless both flags are set. */
cdvs_status cdvs_resize(cdvs_ctx *ctx, int32_t n_images, const uint8_t *const *images,
                        const cdvs_image_desc *sizes, int32_t max_side, uint8_t *out, size_t capacity,
                        cdvs_image_desc *out_sizes, uint32_t flags, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Learned block proposal.  Not in the paper: an extension of its detector
 * (Sec. IV-A, Alg. 1) that predicts, from the 8-bit image, which 16x16 blocks
 * hold interest points, so that the first octave's detection runs only near
 * them.  The network (CDVS_PROPOSAL_PARAMS FP32 parameters, in this order:
 * W1[16][1][3][3], b1[16], W2[16][16][3][3], b2[16], W3[16][16][3][3], b3[16],
 * Wh[16], bh):
 *   x  = (u8 - 128) / 64
 *   A1 = relu(conv3x3(x,  W1, stride 2, pad 1) + b1)   (BF16)
 *   A2 = relu(conv3x3(A1, W2, stride 2, pad 1) + b2)   (BF16)
 *   A3 = relu(conv3x3(A2, W3, stride 1, pad 1) + b3)
 *   logit(block) = Wh . mean over the block's 4x4 cell of A3 + bh
 * conv3x3 is cross-correlation; weights are used in BF16, biases and every
 * sum in FP32.  An image of W x H has ceil(W/16) x ceil(H/16) blocks.
 *
 * With params->use_proposal = 1, cdvs_extract and cdvs_candidates first run
 * the network, then treat each first-octave detection tile (128 x 32 px) in
 * one of three ways: tiles within one block of a proposed block (probability
 * > params->proposal_threshold) run the whole detector, keeping candidates
 * only in their blocks within one block of a proposed block; tiles whose
 * levels a descriptor disc may read store every level without detecting; the
 * rest only build level 3, which the next octave is decimated from.  Later
 * octaves run in full.
 * ------------------------------------------------------------------------- */
#define CDVS_PROPOSAL_PARAMS 4817

/* Copies the network's parameters (host memory, CDVS_PROPOSAL_PARAMS floats)
 * into the context.  INVALID_ARGUMENT when n_params differs. */
cdvs_status cdvs_set_proposal(cdvs_ctx *ctx, const float *params, int32_t n_params);

/* The network's logits for a batch: image i's ceil(W/16) x ceil(H/16) logits,
 * row-major, follow those of images 0..i-1 in logits_out (capacity floats;
 * UNSUPPORTED_SIZE when too small).  Images as in cdvs_extract (flags
 * CDVS_INPUT_DEVICE, CDVS_OUTPUT_DEVICE: logits_out in device memory).
 * Synchronous unless both flags are set. */
cdvs_status cdvs_proposal_logits(cdvs_ctx *ctx, int32_t n_images, const uint8_t *const *images,
                                 const cdvs_image_desc *sizes, float *logits_out, int32_t capacity,
                                 uint32_t flags, void *cuda_stream);

/* One training step of the network on the GPU, every pointer DEVICE memory.
 * images: n_images images of width x height, row pitch `pitch` bytes, back to
 * back.  labels: per block 0 or 1 (same order as the logits), or NULL for a
 * forward pass only.  params: CDVS_PROPOSAL_PARAMS FP32, updated in place by
 * Adam (beta 0.9, 0.999, eps 1e-8, bias correction with `step` >= 1) when
 * lr > 0.  adam_m, adam_v: Adam moments (caller-owned, zero before step 1).
 * grad (CDVS_PROPOSAL_PARAMS) receives the gradient of the mean BCE over all
 * blocks, loss (1 float, may be NULL) the loss, logits (may be NULL) the
 * logits.  bf16 = 1 rounds weights and A1, A2 to BF16 as the inference does;
 * 0 keeps FP32 (gradient checks).  Asynchronous on cuda_stream. */
cdvs_status cdvs_proposal_train_step(cdvs_ctx *ctx, const uint8_t *images, int32_t n_images, int32_t width,
                                     int32_t height, int32_t pitch, const float *labels, float *params,
                                     float *adam_m, float *adam_v, float *grad, float *loss, float *logits,
                                     int32_t step, float lr, int32_t bf16, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * SCFV aggregation (Sec. III-D, Eq. 6-8; the matrix form of Sec. IV-C,
 * Eq. 9-14): for the K descriptors x_t of each image,
 *   y_t = P (x_t - m)                                  (PCA 128 -> 32)
 *   gamma_t(i) = w_i N(y_t; mu_i, diag v_i) / sum_j w_j N(y_t; mu_j, diag v_j)
 *   g_mu(i)    = 1/(K sqrt(w_i))   sum_t gamma_t(i) (y_t - mu_i) / sqrt(v_i)
 *   g_sigma(i) = 1/(K sqrt(2 w_i)) sum_t gamma_t(i) ((y_t - mu_i)^2 / v_i - 1)
 *   delta(i)   = population standard deviation of the 32 entries of g_mu(i)
 * for the 512 components, the components ranked by delta (descending, ties to
 * the lower index), and bit k of the word of each of the first n_select
 * ranked components set when g_mu(i)_k > 0.  An image with no descriptor
 * gives zero gradients.  The two contractions (Eq. 10, and Eq. 12/14's
 * Gamma^T [1 | y | y^2]) run on the tensor cores with operands split in two
 * FP16 halves and three products per term (about 22 significant bits per
 * product, FP32 accumulation; each component's column of Eq. 10's matrix is
 * scaled by a power of two into FP16's range, exactly undone); everything
 * else is FP32.  Should the tensor cores or the copies feeding them not
 * complete within a bounded wait (0.2 s), the affected gradients come out
 * NaN (every image's, when the log-likelihood products time out) and a
 * synchronous call returns CDVS_DEVICE_TIMEOUT; the context stays usable.
 * ------------------------------------------------------------------------- */
#define CDVS_SCFV_COMPONENTS 512
#define CDVS_SCFV_DIM 32

typedef struct {
    const float *pca_mean;   /* 128 */
    const float *pca;        /* 32 x 128, row-major (row j = output dimension j) */
    const float *weights;    /* 512, positive */
    const float *means;      /* 512 x 32 */
    const float *variances;  /* 512 x 32, positive (diagonal) */
} cdvs_scfv_model;

/* Copies a model (host memory) into the context.  INVALID_ARGUMENT unless the
 * weights and variances are positive, the PCA mean has norm <= 2, every
 * PCA row norm <= 64 (an orthonormal PCA has norm 1; the bound keeps the
 * projections of unit descriptors within the range of the FP16 halves) and
 * the derived log-likelihood terms 1/v and mu/v are finite. */
cdvs_status cdvs_set_scfv_model(cdvs_ctx *ctx, const cdvs_scfv_model *model);

/* SCFV of a batch.  desc: the records' descriptors packed over the batch as
 * cdvs_extract writes them (counts[i] rows of 128 floats for image i, in
 * image order; 16-byte aligned in device memory); counts: host memory.
 * Outputs per image (any may be NULL): g_mu and g_sigma [512][32], delta
 * [512], order [512] (component of each rank), bits [n_select] (0 <= n_select
 * <= 512).  flags: CDVS_INPUT_DEVICE (desc on the device), CDVS_OUTPUT_DEVICE
 * (outputs on the device).  Synchronous unless both flags are set.  An
 * asynchronous call returns before its kernels finish and does not read the
 * device status back: a bounded wait that gave up shows only as NaN in g_mu,
 * g_sigma and delta of the affected images, whose order and bits then carry
 * no meaning.  A caller that needs the status as a return value makes a
 * synchronous call. */
cdvs_status cdvs_scfv(cdvs_ctx *ctx, int32_t n_images, const float *desc, const int32_t *counts,
                      int32_t n_select, float *g_mu, float *g_sigma, float *delta, int32_t *order,
                      uint32_t *bits, uint32_t flags, void *cuda_stream);

/* The work shape of interest-point detection (Alg. 1 stages A and B; the
 * same arithmetic in every shape, so results are identical bit for bit).
 * Four variants: 0 and 1 tile the octave in 128 x 32 pixel tiles with one
 * 512-thread CTA per SM, 2 and 3 in 128 x 16 tiles with two 256-thread CTAs
 * per SM; the y pass of the separable filter takes 6, 12, 4 or 10 rows per
 * thread.  variant = -1 (the default) tunes them: while a class of octave
 * launches (the first octave, or the later ones, per storage type and set of
 * filter radii) has a variant without a time, each call runs one such
 * variant and times it with CUDA events on its stream (read back by a later
 * call; first octaves are timed only when the images are on the device, and
 * such calls do not use the CUDA graph); then every octave takes the variant
 * whose time per tile times its tile count for the batch is smallest.
 * variant = 0..3 fixes the shape (the first octave under a block proposal,
 * and octaves whose filter radii exceed 14 (sigma0 above the default), always
 * use variant 0). */
cdvs_status cdvs_set_detect_variant(cdvs_ctx *ctx, int32_t variant);

/* The tuner's state as a JSON object (mode, variant names, per class the
 * measured microseconds per tile of each variant, and the variants of the
 * last call's octaves), NUL-terminated into buf (capacity bytes, may be
 * NULL).  Returns the length of the full text, or -1 for a NULL context. */
int32_t cdvs_detect_tuning(cdvs_ctx *ctx, char *buf, int32_t capacity);

/* Candidate queue capacity per image (candidates of all octaves before the
 * cross-octave check).  0 (the default) sizes it from the image: max(4096,
 * pixels / 16), more than the method finds on any natural image.  When a
 * synchronous call finds more candidates than its queue holds, it runs again
 * with room for every one, so results never depend on which candidates
 * reached the queue first; the context keeps that room for later calls.  An
 * asynchronous call cannot run again: cdvs_wait reports
 * CDVS_CAPACITY_TRUNCATED and later calls get twice the room.  Setting the
 * capacity forgets the room gained so far. */
cdvs_status cdvs_set_candidate_capacity(cdvs_ctx *ctx, int32_t per_image);

/* ---------------------------------------------------------------------------
 * Measurement helper (not part of the method).  Measures the rate of packed
 * FP32 multiply-adds (fma.rn.f32x2, the instruction of interest-point
 * detection's filters and fit) on the context's GPU: a register-only loop on
 * every SM, timed with CUDA events, ~10 ms.  *tflops counts two flops per
 * multiply-add.  Blocks the calling thread; uses a stream of its own.
 * INVALID_ARGUMENT for a NULL argument; CUDA_ERROR if a launch fails.
 */
cdvs_status cdvs_probe_fp32_rate(cdvs_ctx *ctx, double *tflops);

/* ---------------------------------------------------------------------------
 * Testing hook (not part of the method).  The next `count` device workspace
 * allocations of any context in the process fail as cudaMalloc does when the
 * device memory is exhausted: the call that needed them returns
 * CDVS_OUT_OF_MEMORY and leaves its context usable (the workspace is grown
 * again by the next call).  count <= 0 turns the injection off.
 */
void cdvs_inject_alloc_failures(int32_t count);

/* Testing hook (not part of the method).  The next `count` cdvs_scfv calls of
 * any context leave the tensor-core products of the log-likelihoods
 * unissued, so the posterior kernel's bounded wait (0.2 s) runs out with
 * nothing in flight: the call reports DEVICE_TIMEOUT (synchronous calls) and its
 * gradients are NaN; the context stays usable.  count <= 0 turns it off. */
void cdvs_inject_scfv_wait_timeouts(int32_t count);

#ifdef __cplusplus
}
#endif
#endif /* CDVS_H */
