/*
 * cdvs_oracle.h -- plain FP64 CPU statement of the CDVS front end
 * (interest point detection, orientation, 128-D description, and the
 * downstream transform + ternary quantisation) of
 * "Fast MPEG-CDVS Encoder with GPU-CPU Hybrid Computing" (arXiv 1705.09776).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle that the CUDA path is checked
 * against.  It shares no code, header, table or constant generator with the
 * CUDA library, and only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  Nothing here is tuned: every step is a
 * straightforward loop in the order the paper states it.
 *
 * Units: "octave px" are pixels of octave o (pixel i of octave o sits on image
 * pixel 2^o * i); "image px" are pixels of the input image.  Pixel centres
 * are at integer coordinates, origin at the top-left pixel centre.
 */
#ifndef CDVS_ORACLE_H
#define CDVS_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_MAX_OCTAVES 12
#define ORACLE_MAX_SCALES 8
#define ORACLE_MAX_TAPS 129

typedef struct {
    int32_t num_octaves;        /* O: octaves processed at most (Alg. 1 outer loop) */
    int32_t scales_per_octave;  /* K: LoG scales per octave fitted by the cubic (Eq. 2-3) */
    double sigma0;              /* s_0: scale of level 0 of every octave */
    double sigma_in;            /* blur assumed in the input image */
    double contrast_T;          /* |p| threshold at sigma* and after refinement */
    double edge_r;              /* Hessian edge ratio r; reject tr^2/det >= (r+1)^2/r */
    double offset_max;          /* reject a refined offset above this (octave px) */
    double ori_radius;          /* orientation disc radius / sigma (Sec. IV-B: 3.96) */
    double ori_peak_ratio;      /* keep peaks above this fraction of the max (Sec. IV-B: 0.8) */
    double ori_weight_sigma;    /* Gaussian weight std / sigma for the orientation histogram */
    double desc_radius;         /* description disc radius / sigma (Alg. 2: 6) */
    double cell_side;           /* cell side / sigma (Sec. IV-B: 3) */
    double desc_weight_sigma;   /* Gaussian weight std of the descriptor, in cells */
    double dedupe_dlog2;        /* |log2(sigma_a / sigma_b)| window of the cross-octave check */
    int32_t max_keypoints;      /* N kept by the selection step (Eq. 5) */
    int32_t max_orientations;   /* orientation copies kept per keypoint */
    int32_t upright;            /* 1: theta = 0, no orientation stage */
    int32_t pad0;
    /* parity bracketing: 0 for the method itself.  m > 0 accepts every
     * threshold decision that is within a relative m of passing ("loose"),
     * m < 0 rejects every one within |m| of failing ("strict"). */
    double margin;
    /* orientation-bin bracketing, in bins: > 0 moves samples within this
     * distance below a bin boundary up across it, < 0 moves samples within
     * |ori_margin| above a boundary down across it. */
    double ori_margin;
} oracle_params;

/* One interest point (or one (point, orientation) output record). */
typedef struct {
    double x, y, sigma;         /* image px */
    double xo, yo, so;          /* octave px */
    double theta;               /* radians in [0, 2 pi) */
    double response;            /* refined response p-hat */
    double p_ss;                /* d2p/dsigma2 at sigma* (octave px units) */
    double ratio;               /* Hessian tr^2/det */
    int32_t octave, scale_idx;  /* octave o and the level used for description */
    int32_t type;               /* +1 maximum, -1 minimum (in scale and space) */
    int32_t parent;             /* rank of the selected point this record describes */
} oracle_kp;

void oracle_params_default(oracle_params *p);

/* Octave sizes: W_{o+1} = ceil(W_o/2).  Returns the number of octaves
 * processed (both sides >= 3, at most num_octaves); fills Wo/Ho. */
int oracle_octave_dims(int W, int H, const oracle_params *p, int *Wo, int *Ho);
size_t oracle_levels_size(int W, int H, const oracle_params *p);  /* doubles */
size_t oracle_level_offset(int W, int H, const oracle_params *p, int o, int k);

double oracle_scale(const oracle_params *p, int k);        /* s_k, octave px */
double oracle_tau(const oracle_params *p, int o, int k);   /* blur added to the base */
int oracle_gaussian_taps(double tau, double *taps, int cap);  /* returns radius */

void oracle_filter_separable(const double *in, int W, int H, const double *taps, int r,
                             double *out);
void oracle_filter_2d(const double *in, int W, int H, const double *taps, int r, double *out);

/* S1 + S6: all Gaussian levels of all octaves, octave-major then level then
 * row-major.  Returns the number of octaves. */
int oracle_scale_space(const uint8_t *img, int W, int H, int pitch, const oracle_params *p,
                       double *levels);

/* S2: L = s^2 * 5-point Laplacian of G, clamp-to-edge. */
void oracle_laplacian(const double *G, int W, int H, double s, double *L);

/* S3: beta (4 x K, row i = coefficient alpha_i) with alpha = beta * L. */
int oracle_alp_matrix(const oracle_params *p, double *beta);
void oracle_alp_fit(const double *beta, const double *Lk, int K, double alpha[4]);
double oracle_cubic(const double a[4], double s);

/* S4 on one pixel's cubic: 0 none, +1 maximum, -1 minimum. */
int oracle_alp_extremum(const double a[4], const oracle_params *p, double *sigma_star,
                        double *value);

/* S5 on the 3x3 of p(., ., sigma*) (row-major, rows = y).  out: dx, dy,
 * p-hat, ratio.  Returns 1 if the point is kept. */
int oracle_refine(const double q[9], const oracle_params *p, double out[4]);

/* S2-S5 on one octave's K levels: appends candidates, returns their number.
 * *buf is realloc'ed as needed (*cap tracks its size). */
int oracle_detect_octave(const double *levels_o, int W, int H, int o, const oracle_params *p,
                         oracle_kp **buf, int *n, int *cap);

/* S2-S5 on given levels of one octave, candidates copied to out (at most
 * cap); returns their number (a test entry point). */
int oracle_detect_levels(const double *levels_o, int W, int H, int o, const oracle_params *p,
                         oracle_kp *out, int cap);

/* S7: keep[i] = 0 for candidates removed by the cross-octave check. */
void oracle_dedupe(const oracle_kp *c, int n, const oracle_params *p, uint8_t *keep);

/* S8: indices of kept candidates in rank order (at most max_keypoints). */
int oracle_select(const oracle_kp *c, const uint8_t *keep, int n, const oracle_params *p,
                  int *order);

/* S9 histogram alone: h[36] gets the weighted votes of the disc. */
void oracle_orientation_hist(const double *G, int W, int H, double xo, double yo, double so,
                             const oracle_params *p, double *h);
/* S9 peaks of a 36-bin histogram h: up to max_orientations angles in [0, 2 pi). */
int oracle_orientation_peaks(const double *h, const oracle_params *p, double *thetas);
/* S10 votes alone: the 128 unnormalised trilinear sums. */
void oracle_descriptor_hist(const double *G, int W, int H, double xo, double yo, double so,
                            double theta, const oracle_params *p, double *d);
/* S9: orientation histogram (36 bins) and up to max_orientations peaks. */
int oracle_orientations(const double *G, int W, int H, double xo, double yo, double so,
                        const oracle_params *p, double *thetas, double *hist36);

/* S10: 128-D descriptor, cells row-major (y, x), 8 bins fastest. */
void oracle_descriptor(const double *G, int W, int H, double xo, double yo, double so,
                       double theta, const oracle_params *p, double *desc128);

/* Description level index for a point of scale so (octave px). */
int oracle_desc_level(const oracle_params *p, double so);

/* S1-S10 on one image.  Writes at most cap records; returns the number of
 * records the method produces (may exceed cap).  n_candidates (may be NULL)
 * gets the number of refined candidates before the cross-octave check. */
int oracle_extract(const uint8_t *img, int W, int H, int pitch, const oracle_params *p,
                   oracle_kp *kp_out, double *desc_out, int cap, int *n_candidates);

/* S1-S5 only: all refined candidates of all octaves (before S7). */
int oracle_candidates(const uint8_t *img, int W, int H, int pitch, const oracle_params *p,
                      oracle_kp *out, int cap);

/* S7-S8 on given candidates: writes the selected indices in rank order. */
int oracle_dedupe_select(const oracle_kp *c, int n, const oracle_params *p, int *order);

/* S9-S10 for given points (octave, xo, yo, so taken from each record). */
int oracle_describe(const uint8_t *img, int W, int H, int pitch, const oracle_params *p,
                    const oracle_kp *pts, int n_pts, oracle_kp *kp_out, double *desc_out,
                    int cap);

/* oracle_extract over a batch, image-parallel on n_threads threads.
 * Record i of image b goes to kp_out[b * cap + i]. */
int oracle_extract_batch(int n, const uint8_t *const *imgs, const int *W, const int *H,
                         const int *pitch, const oracle_params *p, oracle_kp *kp_out,
                         double *desc_out, int cap, int *counts, int n_threads);

/* Threads an image-parallel batch uses by default. */
int oracle_num_threads(void);

/* S11: order-8 transforms of each cell histogram (set A when cx + cy is even,
 * set B otherwise) and ternary quantisation with per-element thresholds. */
void oracle_transform(const double *desc128, double *v128);
void oracle_ternary(const double *v128, const double *t_lo, const double *t_hi, int8_t *q);

#ifdef __cplusplus
}
#endif
#endif
