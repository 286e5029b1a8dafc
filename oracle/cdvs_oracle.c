/*
 * cdvs_oracle.c -- plain FP64 CPU oracle of the CDVS front end of
 * "Fast MPEG-CDVS Encoder with GPU-CPU Hybrid Computing" (arXiv 1705.09776).
 *
 * TEST INFRASTRUCTURE ONLY (see cdvs_oracle.h).  Slow on purpose: serial
 * loops, clamp-to-edge borders, no tiling, no fusion.  Each function names
 * the passage of the paper it follows; where the paper is silent the reading
 * taken is stated beside the code.
 */
#include "cdvs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

void oracle_params_default(oracle_params *p) {
    memset(p, 0, sizeof(*p));
    p->num_octaves = 4;
    p->scales_per_octave = 4;
    p->sigma0 = 1.6;
    p->sigma_in = 0.5;
    p->contrast_T = 4.0;
    p->edge_r = 10.0;
    p->offset_max = 0.5;
    p->ori_radius = 3.96;      /* Sec. IV-B: neighbourhood radius 3.96 sigma */
    p->ori_peak_ratio = 0.8;   /* Sec. IV-B: bins above 0.8 of the highest peak */
    p->ori_weight_sigma = 1.5;
    p->desc_radius = 6.0;      /* Alg. 2 stage B: distance < 6 sigma */
    p->cell_side = 3.0;        /* Sec. IV-B: cell side 3 sigma */
    p->desc_weight_sigma = 2.0;
    p->dedupe_dlog2 = 1.0 / 3.0;
    p->max_keypoints = 300;    /* Sec. III-B: around 300 selected features */
    p->max_orientations = 4;
    p->upright = 0;
    p->margin = 0.0;
    p->ori_margin = 0.0;
}

/* ---------------------------------------------------------------- octaves */

int oracle_octave_dims(int W, int H, const oracle_params *p, int *Wo, int *Ho) {
    int n = 0, w = W, h = H;
    for (int o = 0; o < p->num_octaves && o < ORACLE_MAX_OCTAVES; ++o) {
        if (w < 3 || h < 3) break;
        Wo[o] = w;
        Ho[o] = h;
        ++n;
        w = (w + 1) / 2; /* ceil(W/2): decimation keeps the even coordinates */
        h = (h + 1) / 2;
    }
    return n;
}

size_t oracle_levels_size(int W, int H, const oracle_params *p) {
    int Wo[ORACLE_MAX_OCTAVES], Ho[ORACLE_MAX_OCTAVES];
    int O = oracle_octave_dims(W, H, p, Wo, Ho);
    size_t s = 0;
    for (int o = 0; o < O; ++o) s += (size_t)p->scales_per_octave * Wo[o] * Ho[o];
    return s;
}

size_t oracle_level_offset(int W, int H, const oracle_params *p, int o, int k) {
    int Wo[ORACLE_MAX_OCTAVES], Ho[ORACLE_MAX_OCTAVES];
    oracle_octave_dims(W, H, p, Wo, Ho);
    size_t s = 0;
    for (int i = 0; i < o; ++i) s += (size_t)p->scales_per_octave * Wo[i] * Ho[i];
    return s + (size_t)k * Wo[o] * Ho[o];
}

/* ------------------------------------------------------ S1: Gaussian levels */

/* s_k = sigma0 * 2^(k/(K-1)): K levels spanning one octave [sigma0, 2 sigma0]. */
double oracle_scale(const oracle_params *p, int k) {
    return p->sigma0 * pow(2.0, (double)k / (double)(p->scales_per_octave - 1));
}

/* Every level is filtered directly from the octave base (Alg. 1, stage A:
 * T_k and G_{o,k} both use the base G_{o,0} and the kernel g_k).  The base of
 * octave 0 is the input, assumed blurred by sigma_in; the base of octave
 * o >= 1 is the decimated top level, blurred by sigma0 in its own pixels.
 * The added blur is tau = sqrt(s_k^2 - base^2) (Gaussians compose by adding
 * variances). */
double oracle_tau(const oracle_params *p, int o, int k) {
    double s = oracle_scale(p, k);
    double b = (o == 0) ? p->sigma_in : p->sigma0;
    double v = s * s - b * b;
    return v > 0.0 ? sqrt(v) : 0.0;
}

/* Sampled Gaussian of std tau on [-r, r], r = ceil(4 tau), divided by its
 * sum; tau = 0 gives the identity. */
int oracle_gaussian_taps(double tau, double *taps, int cap) {
    if (tau <= 0.0) {
        if (cap >= 1) taps[0] = 1.0;
        return 0;
    }
    int r = (int)ceil(4.0 * tau);
    if (2 * r + 1 > cap) return -1;
    double sum = 0.0;
    for (int i = -r; i <= r; ++i) {
        taps[i + r] = exp(-(double)(i * i) / (2.0 * tau * tau));
        sum += taps[i + r];
    }
    for (int i = 0; i < 2 * r + 1; ++i) taps[i] /= sum;
    return r;
}

/* Eq. 1 / Alg. 1: first pass along the first index (rows i+p), second pass
 * along the second index (columns j+p); borders clamp to the edge. */
void oracle_filter_separable(const double *in, int W, int H, const double *taps, int r,
                             double *out) {
    double *t = (double *)malloc(sizeof(double) * (size_t)W * H);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int q = -r; q <= r; ++q) acc += in[(size_t)clampi(i + q, 0, H - 1) * W + j] * taps[q + r];
            t[(size_t)i * W + j] = acc;
        }
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int q = -r; q <= r; ++q) acc += t[(size_t)i * W + clampi(j + q, 0, W - 1)] * taps[q + r];
            out[(size_t)i * W + j] = acc;
        }
    free(t);
}

/* Brute-force 2-D convolution with the outer-product kernel (self-test only). */
void oracle_filter_2d(const double *in, int W, int H, const double *taps, int r, double *out) {
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int a = -r; a <= r; ++a)
                for (int b = -r; b <= r; ++b)
                    acc += in[(size_t)clampi(i + a, 0, H - 1) * W + clampi(j + b, 0, W - 1)] *
                           taps[a + r] * taps[b + r];
            out[(size_t)i * W + j] = acc;
        }
}

/* Alg. 1: G_{0,0} = I; for each octave, every level from the base; then
 * G_{o+1,0} = Downsample(top level): decimation at even coordinates (S6). */
int oracle_scale_space(const uint8_t *img, int W, int H, int pitch, const oracle_params *p,
                       double *levels) {
    int Wo[ORACLE_MAX_OCTAVES], Ho[ORACLE_MAX_OCTAVES];
    int O = oracle_octave_dims(W, H, p, Wo, Ho);
    const int K = p->scales_per_octave;
    double *base = (double *)malloc(sizeof(double) * (size_t)W * H);
    double taps[ORACLE_MAX_TAPS];
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) base[(size_t)y * W + x] = (double)img[(size_t)y * pitch + x];
    size_t off = 0;
    for (int o = 0; o < O; ++o) {
        const int w = Wo[o], h = Ho[o];
        if (o > 0) {
            const double *top = levels + off - (size_t)Wo[o - 1] * Ho[o - 1];
            for (int y = 0; y < h; ++y)
                for (int x = 0; x < w; ++x)
                    base[(size_t)y * w + x] = top[(size_t)(2 * y) * Wo[o - 1] + 2 * x];
        }
        for (int k = 0; k < K; ++k) {
            int r = oracle_gaussian_taps(oracle_tau(p, o, k), taps, ORACLE_MAX_TAPS);
            oracle_filter_separable(base, w, h, taps, r, levels + off);
            off += (size_t)w * h;
        }
    }
    free(base);
    return O;
}

/* ------------------------------------------------------------------ S2 LoG */

/* Alg. 1: L_{o,k} = sum over the 3x3 of G_{o,k} * f; f is the 5-point
 * Laplacian, scaled by s_k^2 to give the scale-normalised response. */
void oracle_laplacian(const double *G, int W, int H, double s, double *L) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double c = G[(size_t)y * W + x];
            double l = G[(size_t)y * W + clampi(x - 1, 0, W - 1)];
            double r = G[(size_t)y * W + clampi(x + 1, 0, W - 1)];
            double u = G[(size_t)clampi(y - 1, 0, H - 1) * W + x];
            double d = G[(size_t)clampi(y + 1, 0, H - 1) * W + x];
            L[(size_t)y * W + x] = s * s * (l + r + u + d - 4.0 * c);
        }
}

/* ------------------------------------------------------------------ S3 ALP */

/* Eq. 2-3: p(sigma) = sum_i alpha_i sigma^i with alpha_i = sum_k beta_{k,i} L_k.
 * beta is the least-squares fit of a cubic to the K samples (L_k at s_k):
 * beta = (V^T V)^-1 V^T with V_{k,i} = s_k^i; for K = 4 this is V^-1, the
 * exact interpolating cubic.  Solved by Gauss-Jordan with partial pivoting. */
int oracle_alp_matrix(const oracle_params *p, double *beta) {
    const int K = p->scales_per_octave;
    double V[ORACLE_MAX_SCALES][4];
    for (int k = 0; k < K; ++k) {
        double s = oracle_scale(p, k), v = 1.0;
        for (int i = 0; i < 4; ++i) {
            V[k][i] = v;
            v *= s;
        }
    }
    /* augmented system [V^T V | V^T] */
    double A[4][4 + ORACLE_MAX_SCALES];
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += V[k][i] * V[k][j];
            A[i][j] = acc;
        }
        for (int k = 0; k < K; ++k) A[i][4 + k] = V[k][i];
    }
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int i = c + 1; i < 4; ++i)
            if (fabs(A[i][c]) > fabs(A[piv][c])) piv = i;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int j = 0; j < 4 + K; ++j) {
                double t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        double d = A[c][c];
        for (int j = 0; j < 4 + K; ++j) A[c][j] /= d;
        for (int i = 0; i < 4; ++i) {
            if (i == c) continue;
            double f = A[i][c];
            if (f != 0.0)
                for (int j = 0; j < 4 + K; ++j) A[i][j] -= f * A[c][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < K; ++k) beta[i * K + k] = A[i][4 + k];
    return 0;
}

void oracle_alp_fit(const double *beta, const double *Lk, int K, double alpha[4]) {
    for (int i = 0; i < 4; ++i) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += beta[i * K + k] * Lk[k];
        alpha[i] = acc;
    }
}

double oracle_cubic(const double a[4], double s) { return ((a[3] * s + a[2]) * s + a[1]) * s + a[0]; }

/* ------------------------------------------------------ S4: ALP extremum */

/* Sec. III-A (ALP): the extremum scales are the roots of dp/dsigma =
 * 3 a3 s^2 + 2 a2 s + a1 = 0, solved in the cancellation-free form
 * q = -(B + sign(B) sqrt(D))/2, roots q/A and C/q.  A root counts if it lies
 * in [s_0, s_{K-1}], p'' != 0 there, and |p| >= T; p'' < 0 makes it a maximum,
 * p'' > 0 a minimum.  When both roots count, the larger |p| wins (ties: the
 * smaller sigma).  |a3| below 1e-12 of sum |a| is treated as a quadratic p
 * (one root of the linear derivative). */
int oracle_alp_extremum(const double a[4], const oracle_params *p, double *sigma_star,
                        double *value) {
    const double m = p->margin;
    const double lo = oracle_scale(p, 0) * (1.0 - m);
    const double hi = oracle_scale(p, p->scales_per_octave - 1) * (1.0 + m);
    const double T = p->contrast_T * (1.0 - m);
    double sumabs = fabs(a[0]) + fabs(a[1]) + fabs(a[2]) + fabs(a[3]);
    if (sumabs == 0.0) return 0;
    double A = 3.0 * a[3], B = 2.0 * a[2], C = a[1];
    double roots[2];
    int nr = 0;
    if (fabs(a[3]) < 1e-12 * sumabs) {
        if (B != 0.0) roots[nr++] = -C / B;
    } else {
        double D = B * B - 4.0 * A * C;
        if (D <= 0.0) return 0; /* no real root, or a double root (inflection) */
        double q = -0.5 * (B + copysign(sqrt(D), B));
        roots[nr++] = q / A;
        if (q != 0.0) roots[nr++] = C / q;
    }
    int best_t = 0;
    double best_s = 0.0, best_v = 0.0;
    for (int i = 0; i < nr; ++i) {
        double s = roots[i];
        if (!(s >= lo && s <= hi)) continue;
        double pdd = 6.0 * a[3] * s + 2.0 * a[2];
        if (pdd == 0.0) continue;
        double v = oracle_cubic(a, s);
        if (!(fabs(v) >= T)) continue;
        int t = pdd < 0.0 ? +1 : -1;
        if (best_t == 0 || fabs(v) > fabs(best_v) || (fabs(v) == fabs(best_v) && s < best_s)) {
            best_t = t;
            best_s = s;
            best_v = v;
        }
    }
    if (best_t) {
        *sigma_star = best_s;
        *value = best_v;
    }
    return best_t;
}

/* ------------------------------------------------------ S5: refinement */

/* Alg. 1 stage B (CoordinateRefine) on the 3x3 of p(., ., sigma*): central
 * differences give the gradient g and Hessian H; the interpolated offset is
 * delta = -H^-1 g, the interpolated response p + g.delta/2.  Unstable points
 * are dropped: det H <= 0, tr^2/det >= (r+1)^2/r, |delta| > offset_max, or
 * |p-hat| < T. */
int oracle_refine(const double q[9], const oracle_params *p, double out[4]) {
    const double m = p->margin;
    double gx = 0.5 * (q[5] - q[3]);
    double gy = 0.5 * (q[7] - q[1]);
    double hxx = q[5] - 2.0 * q[4] + q[3];
    double hyy = q[7] - 2.0 * q[4] + q[1];
    double hxy = 0.25 * (q[8] - q[6] - q[2] + q[0]);
    double det = hxx * hyy - hxy * hxy;
    if (!(det > 0.0)) return 0;
    double tr = hxx + hyy;
    double ratio = tr * tr / det;
    double lim = (p->edge_r + 1.0) * (p->edge_r + 1.0) / p->edge_r;
    if (!(ratio < lim * (1.0 + m))) return 0;
    double dx = -(hyy * gx - hxy * gy) / det;
    double dy = -(hxx * gy - hxy * gx) / det;
    double omax = p->offset_max * (1.0 + m);
    if (!(fabs(dx) <= omax && fabs(dy) <= omax)) return 0;
    double ph = q[4] + 0.5 * (gx * dx + gy * dy);
    if (!(fabs(ph) >= p->contrast_T * (1.0 - m))) return 0;
    out[0] = dx;
    out[1] = dy;
    out[2] = ph;
    out[3] = ratio;
    return 1;
}

/* ------------------------------------------------ S2-S5 on one octave */

static void push_kp(oracle_kp **buf, int *n, int *cap, const oracle_kp *k) {
    if (*n >= *cap) {
        *cap = *cap ? 2 * *cap : 1024;
        *buf = (oracle_kp *)realloc(*buf, sizeof(oracle_kp) * (size_t)*cap);
    }
    (*buf)[(*n)++] = *k;
}

/* Alg. 1 stage A (LoG + ALP extremum per pixel, compared with its 8
 * neighbours: each neighbour's cubic evaluated at the centre's sigma* must be
 * strictly below it for a maximum, strictly above for a minimum) and stage B.
 * Pixels on the octave border have no 8 neighbours and are not tested. */
int oracle_detect_octave(const double *levels_o, int W, int H, int o, const oracle_params *p,
                         oracle_kp **buf, int *n, int *cap) {
    const int K = p->scales_per_octave;
    const size_t np = (size_t)W * H;
    const double m = p->margin;
    double beta[4 * ORACLE_MAX_SCALES];
    if (oracle_alp_matrix(p, beta)) return 0;
    double *L = (double *)malloc(sizeof(double) * np * K);
    double *al = (double *)malloc(sizeof(double) * np * 4);
    for (int k = 0; k < K; ++k) oracle_laplacian(levels_o + k * np, W, H, oracle_scale(p, k), L + k * np);
    for (size_t i = 0; i < np; ++i) {
        double Lk[ORACLE_MAX_SCALES];
        for (int k = 0; k < K; ++k) Lk[k] = L[k * np + i];
        oracle_alp_fit(beta, Lk, K, al + 4 * i);
    }
    const double scale = ldexp(1.0, o);
    int found = 0;
    for (int y = 1; y < H - 1; ++y)
        for (int x = 1; x < W - 1; ++x) {
            double ss, v;
            int t = oracle_alp_extremum(al + 4 * ((size_t)y * W + x), p, &ss, &v);
            if (!t) continue;
            double q[9];
            int ok = 1;
            for (int dy = -1; dy <= 1 && ok; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    double pn = oracle_cubic(al + 4 * ((size_t)(y + dy) * W + (x + dx)), ss);
                    q[(dy + 1) * 3 + (dx + 1)] = pn;
                    if (dx == 0 && dy == 0) continue;
                    if (t > 0 ? !(pn < v + m * fabs(v)) : !(pn > v - m * fabs(v))) {
                        ok = 0;
                        break;
                    }
                }
            if (!ok) continue;
            q[4] = v;
            double r[4];
            if (!oracle_refine(q, p, r)) continue;
            oracle_kp k;
            memset(&k, 0, sizeof(k));
            k.xo = x + r[0];
            k.yo = y + r[1];
            k.so = ss;
            k.x = k.xo * scale;
            k.y = k.yo * scale;
            k.sigma = ss * scale;
            const double *a = al + 4 * ((size_t)y * W + x);
            k.response = r[2];
            k.p_ss = 6.0 * a[3] * ss + 2.0 * a[2];
            k.ratio = r[3];
            k.octave = o;
            k.scale_idx = oracle_desc_level(p, ss);
            k.type = t;
            k.parent = -1;
            push_kp(buf, n, cap, &k);
            ++found;
        }
    free(L);
    free(al);
    return found;
}

/* Stages S2-S5 on one octave's given levels (K planes of W x H, level k at
 * k W H), with its candidates copied to out (at most cap).  Returns their
 * count.  A test entry point: it lets a test build levels whose responses tie
 * exactly, which filtered images do not give. */
int oracle_detect_levels(const double *levels_o, int W, int H, int o, const oracle_params *p,
                         oracle_kp *out, int cap) {
    oracle_kp *buf = NULL;
    int n = 0, bcap = 0;
    oracle_detect_octave(levels_o, W, H, o, p, &buf, &n, &bcap);
    for (int i = 0; i < n && i < cap; ++i) out[i] = buf[i];
    free(buf);
    return n;
}

/* ------------------------------------------------ S7: cross-octave check */

/* Alg. 1 stage C: candidates of adjacent octaves that are close in (x, y,
 * sigma) -- |dx|, |dy| within one pixel of the coarser octave and
 * |log2(sigma_a/sigma_b)| within dedupe_dlog2 -- are duplicates, and the one
 * with the lower |response| is removed.  All pairs are decided at once on the
 * original set; equal |response| removes the coarser one.  O(n^2) scan. */
void oracle_dedupe(const oracle_kp *c, int n, const oracle_params *p, uint8_t *keep) {
    const double m = p->margin;
    for (int a = 0; a < n; ++a) {
        keep[a] = 1;
        double ra = fabs(c[a].response);
        for (int b = 0; b < n; ++b) {
            int d = c[a].octave - c[b].octave;
            if (d != 1 && d != -1) continue;
            int oc = c[a].octave > c[b].octave ? c[a].octave : c[b].octave;
            double win = ldexp(1.0, oc) * (1.0 - m);
            if (!(fabs(c[a].x - c[b].x) <= win && fabs(c[a].y - c[b].y) <= win)) continue;
            if (!(fabs(log2(c[a].sigma / c[b].sigma)) <= p->dedupe_dlog2 * (1.0 - m))) continue;
            double rb = fabs(c[b].response);
            if (rb > ra * (1.0 + m) || (m == 0.0 && rb == ra && c[b].octave < c[a].octave)) {
                keep[a] = 0;
                break;
            }
        }
    }
}

/* ------------------------------------------------ S8: selection */

static const oracle_kp *g_sel_c;
static int sel_cmp(const void *pa, const void *pb) {
    const oracle_kp *a = g_sel_c + *(const int *)pa, *b = g_sel_c + *(const int *)pb;
    double ra = fabs(a->response), rb = fabs(b->response);
    if (ra != rb) return ra > rb ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    if (a->sigma != b->sigma) return a->sigma < b->sigma ? -1 : 1;
    if (a->octave != b->octave) return a->octave < b->octave ? -1 : 1;
    return 0;
}

/* Eq. 5: rank by relevance and keep the first N.  The normative relevance
 * tables f1..f5 are not available; |p-hat| stands in for r.  Ties are broken
 * by (y, x, sigma, octave) ascending, so the order is total. */
int oracle_select(const oracle_kp *c, const uint8_t *keep, int n, const oracle_params *p,
                  int *order) {
    int *idx = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (keep[i]) idx[m++] = i;
    /* qsort is not stable, but sel_cmp is a total order on distinct points */
#ifdef _OPENMP
#pragma omp critical(oracle_sel)
#endif
    {
        g_sel_c = c;
        qsort(idx, (size_t)m, sizeof(int), sel_cmp);
    }
    int N = m < p->max_keypoints ? m : p->max_keypoints;
    memcpy(order, idx, sizeof(int) * (size_t)N);
    free(idx);
    return N;
}

/* ------------------------------------------------ S9: orientation */

int oracle_desc_level(const oracle_params *p, double so) {
    const int K = p->scales_per_octave;
    int k = (int)lround((double)(K - 1) * log2(so / p->sigma0));
    return clampi(k, 0, K - 1);
}

static inline void gradient(const double *G, int W, int H, int u, int v, double *gx, double *gy) {
    *gx = G[(size_t)v * W + clampi(u + 1, 0, W - 1)] - G[(size_t)v * W + clampi(u - 1, 0, W - 1)];
    *gy = G[(size_t)clampi(v + 1, 0, H - 1) * W + u] - G[(size_t)clampi(v - 1, 0, H - 1) * W + u];
}

/* Sec. IV-B / Alg. 2 stage A, the histogram: gradients of the pixels closer
 * than ori_radius * sigma vote, with weight |g| * exp(-d^2 / (2 (w sigma)^2)),
 * w = ori_weight_sigma, into 36 bins of atan2(gy, gx) (bin b covers angles
 * [b, b + 1) * 2 pi / 36, hard assignment, no smoothing). */
void oracle_orientation_hist(const double *G, int W, int H, double xo, double yo, double so,
                             const oracle_params *p, double *h) {
    const double m = p->margin;
    memset(h, 0, sizeof(double) * 36);
    /* the disc membership (distance < ori_radius * sigma) is a threshold
     * decision too: the bracketing runs move the radius by the margin */
    const double R = p->ori_radius * so * (1.0 + m), R2 = R * R;
    const double sw = p->ori_weight_sigma * so;
    for (int v = (int)ceil(yo - R); v <= (int)floor(yo + R); ++v) {
        if (v < 0 || v >= H) continue;
        for (int u = (int)ceil(xo - R); u <= (int)floor(xo + R); ++u) {
            if (u < 0 || u >= W) continue;
            double d2 = (u - xo) * (u - xo) + (v - yo) * (v - yo);
            if (!(d2 < R2)) continue;
            double gx, gy;
            gradient(G, W, H, u, v, &gx, &gy);
            double w = sqrt(gx * gx + gy * gy) * exp(-d2 / (2.0 * sw * sw));
            double f = 36.0 * atan2(gy, gx) / (2.0 * M_PI);
            double fl = floor(f);
            int b = (int)fl;
            double frac = f - fl;
            if (p->ori_margin > 0.0 && frac > 1.0 - p->ori_margin) b += 1;
            if (p->ori_margin < 0.0 && frac < -p->ori_margin) b -= 1;
            b = ((b % 36) + 36) % 36;
            h[b] += w;
        }
    }
}

/* Sec. IV-B / Alg. 2 stage A, the peaks: every bin that is a local maximum
 * (strictly above both circular neighbours) and above ori_peak_ratio times
 * the highest bin gives an orientation, refined to the vertex of the parabola
 * through the bin and its two neighbours (bin centres at b + 1/2).  At most
 * max_orientations are returned, by bin value descending, ties by bin index
 * ascending. */
int oracle_orientation_peaks(const double *h, const oracle_params *p, double *thetas) {
    const double m = p->margin;
    double mx = 0.0;
    for (int b = 0; b < 36; ++b) mx = h[b] > mx ? h[b] : mx;
    double pv[36], pt[36];
    int pb[36], np = 0;
    for (int b = 0; b < 36; ++b) {
        double l = h[(b + 35) % 36], c = h[b], r = h[(b + 1) % 36];
        if (!(c > l && c > r)) continue;
        if (!(c > p->ori_peak_ratio * mx * (1.0 - m))) continue;
        double off = 0.5 * (l - r) / (l - 2.0 * c + r);
        double th = 2.0 * M_PI * ((double)b + 0.5 + off) / 36.0;
        th = fmod(th, 2.0 * M_PI);
        if (th < 0.0) th += 2.0 * M_PI;
        pv[np] = c;
        pt[np] = th;
        pb[np] = b;
        ++np;
    }
    /* order by bin value descending, ties by bin index ascending */
    for (int i = 1; i < np; ++i)
        for (int j = i; j > 0 && (pv[j] > pv[j - 1] || (pv[j] == pv[j - 1] && pb[j] < pb[j - 1])); --j) {
            double tv = pv[j]; pv[j] = pv[j - 1]; pv[j - 1] = tv;
            double tt = pt[j]; pt[j] = pt[j - 1]; pt[j - 1] = tt;
            int tb = pb[j]; pb[j] = pb[j - 1]; pb[j - 1] = tb;
        }
    int n = np < p->max_orientations ? np : p->max_orientations;
    for (int i = 0; i < n; ++i) thetas[i] = pt[i];
    return n;
}

/* Sec. IV-B / Alg. 2 stage A: the histogram, then its peaks. */
int oracle_orientations(const double *G, int W, int H, double xo, double yo, double so,
                        const oracle_params *p, double *thetas, double *hist36) {
    double h[36];
    oracle_orientation_hist(G, W, H, xo, yo, so, p, h);
    if (hist36) memcpy(hist36, h, sizeof(h));
    return oracle_orientation_peaks(h, p, thetas);
}

/* ------------------------------------------------ S10: descriptor */

/* Sec. IV-B / Alg. 2 stage B, the votes: the pixels closer than
 * desc_radius * sigma are rotated by -theta into a 4 x 4 grid of cells of
 * side cell_side * sigma; each gradient (angle relative to theta) is spread
 * trilinearly over the two nearest cells in x and y and the two nearest of 8
 * orientation bins, with weight |g| * exp(-(u^2 + v^2) / (2 desc_weight_sigma^2)),
 * (u, v) in cells.  h gets the 128 unnormalised sums, cells row-major (y, x),
 * 8 bins fastest. */
void oracle_descriptor_hist(const double *G, int W, int H, double xo, double yo, double so,
                            double theta, const oracle_params *p, double *d) {
    memset(d, 0, sizeof(double) * 128);
    /* disc membership (distance < desc_radius * sigma), bracketed like every
     * other threshold decision */
    const double R = p->desc_radius * so * (1.0 + p->margin), R2 = R * R;
    const double cs = p->cell_side * so;
    const double ct = cos(theta), st = sin(theta);
    const double ws2 = 2.0 * p->desc_weight_sigma * p->desc_weight_sigma;
    for (int v = (int)ceil(yo - R); v <= (int)floor(yo + R); ++v) {
        if (v < 0 || v >= H) continue;
        for (int u = (int)ceil(xo - R); u <= (int)floor(xo + R); ++u) {
            if (u < 0 || u >= W) continue;
            double du = u - xo, dv = v - yo;
            if (!(du * du + dv * dv < R2)) continue;
            double xr = (ct * du + st * dv) / cs;
            double yr = (-st * du + ct * dv) / cs;
            double gx, gy;
            gradient(G, W, H, u, v, &gx, &gy);
            double mag = sqrt(gx * gx + gy * gy);
            double rel = atan2(gy, gx) - theta;
            rel = fmod(rel, 2.0 * M_PI);
            if (rel < 0.0) rel += 2.0 * M_PI;
            double ob = 8.0 * rel / (2.0 * M_PI);
            if (ob >= 8.0) ob -= 8.0;
            double w = mag * exp(-(xr * xr + yr * yr) / ws2);
            double cx = xr + 1.5, cy = yr + 1.5;
            double x0 = floor(cx), y0 = floor(cy), o0 = floor(ob);
            double fx = cx - x0, fy = cy - y0, fo = ob - o0;
            for (int iy = 0; iy < 2; ++iy) {
                int yy = (int)y0 + iy;
                if (yy < 0 || yy > 3) continue;
                double wy = iy ? fy : 1.0 - fy;
                for (int ix = 0; ix < 2; ++ix) {
                    int xx = (int)x0 + ix;
                    if (xx < 0 || xx > 3) continue;
                    double wx = ix ? fx : 1.0 - fx;
                    for (int io = 0; io < 2; ++io) {
                        int oo = ((int)o0 + io) % 8;
                        double wo = io ? fo : 1.0 - fo;
                        d[(yy * 4 + xx) * 8 + oo] += w * wy * wx * wo;
                    }
                }
            }
        }
    }
}

/* Sec. IV-B / Alg. 2 stage B: the votes, then the 128 values L2-normalised,
 * clamped at 0.2 and renormalised. */
void oracle_descriptor(const double *G, int W, int H, double xo, double yo, double so,
                       double theta, const oracle_params *p, double *d) {
    oracle_descriptor_hist(G, W, H, xo, yo, so, theta, p, d);
    double n2 = 0.0;
    for (int i = 0; i < 128; ++i) n2 += d[i] * d[i];
    if (n2 <= 0.0) return;
    double inv = 1.0 / sqrt(n2);
    n2 = 0.0;
    for (int i = 0; i < 128; ++i) {
        d[i] *= inv;
        if (d[i] > 0.2) d[i] = 0.2;
        n2 += d[i] * d[i];
    }
    inv = 1.0 / sqrt(n2);
    for (int i = 0; i < 128; ++i) d[i] *= inv;
}

/* ------------------------------------------------ pipeline */

static int all_candidates(const double *levels, int W, int H, const oracle_params *p,
                          oracle_kp **buf, int *cap) {
    int Wo[ORACLE_MAX_OCTAVES], Ho[ORACLE_MAX_OCTAVES];
    int O = oracle_octave_dims(W, H, p, Wo, Ho);
    int n = 0;
    size_t off = 0;
    for (int o = 0; o < O; ++o) {
        oracle_detect_octave(levels + off, Wo[o], Ho[o], o, p, buf, &n, cap);
        off += (size_t)p->scales_per_octave * Wo[o] * Ho[o];
    }
    return n;
}

static int describe_points(const double *levels, int W, int H, const oracle_params *p,
                           const oracle_kp *pts, int n_pts, oracle_kp *kp_out,
                           double *desc_out, int cap) {
    int total = 0;
    for (int i = 0; i < n_pts; ++i) {
        const oracle_kp *s = pts + i;
        int o = s->octave;
        int k = oracle_desc_level(p, s->so);
        int Wo[ORACLE_MAX_OCTAVES], Ho[ORACLE_MAX_OCTAVES];
        int O = oracle_octave_dims(W, H, p, Wo, Ho);
        if (o < 0 || o >= O) continue;
        const double *G = levels + oracle_level_offset(W, H, p, o, k);
        double th[36];
        int nt;
        if (p->upright) {
            th[0] = 0.0;
            nt = 1;
        } else {
            oracle_params q = *p;
            if (q.max_orientations > 36) q.max_orientations = 36;
            nt = oracle_orientations(G, Wo[o], Ho[o], s->xo, s->yo, s->so, &q, th, NULL);
        }
        for (int j = 0; j < nt; ++j) {
            if (total < cap) {
                oracle_kp r = *s;
                r.theta = th[j];
                r.scale_idx = k;
                r.parent = i;
                kp_out[total] = r;
                oracle_descriptor(G, Wo[o], Ho[o], s->xo, s->yo, s->so, th[j], p,
                                  desc_out + (size_t)total * 128);
            }
            ++total;
        }
    }
    return total;
}

int oracle_candidates(const uint8_t *img, int W, int H, int pitch, const oracle_params *p,
                      oracle_kp *out, int cap) {
    double *levels = (double *)malloc(sizeof(double) * oracle_levels_size(W, H, p));
    oracle_scale_space(img, W, H, pitch, p, levels);
    oracle_kp *buf = NULL;
    int bcap = 0;
    int n = all_candidates(levels, W, H, p, &buf, &bcap);
    for (int i = 0; i < n && i < cap; ++i) out[i] = buf[i];
    free(buf);
    free(levels);
    return n;
}

int oracle_dedupe_select(const oracle_kp *c, int n, const oracle_params *p, int *order) {
    uint8_t *keep = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    oracle_dedupe(c, n, p, keep);
    int N = oracle_select(c, keep, n, p, order);
    free(keep);
    return N;
}

int oracle_describe(const uint8_t *img, int W, int H, int pitch, const oracle_params *p,
                    const oracle_kp *pts, int n_pts, oracle_kp *kp_out, double *desc_out,
                    int cap) {
    double *levels = (double *)malloc(sizeof(double) * oracle_levels_size(W, H, p));
    oracle_scale_space(img, W, H, pitch, p, levels);
    int total = describe_points(levels, W, H, p, pts, n_pts, kp_out, desc_out, cap);
    free(levels);
    return total;
}

/* Alg. 1 then Alg. 2 on one image, with the selection of Eq. 5 between them. */
int oracle_extract(const uint8_t *img, int W, int H, int pitch, const oracle_params *p,
                   oracle_kp *kp_out, double *desc_out, int cap, int *n_candidates) {
    double *levels = (double *)malloc(sizeof(double) * oracle_levels_size(W, H, p));
    oracle_scale_space(img, W, H, pitch, p, levels);
    oracle_kp *cand = NULL;
    int ccap = 0;
    int n = all_candidates(levels, W, H, p, &cand, &ccap);
    if (n_candidates) *n_candidates = n;
    int *order = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int N = oracle_dedupe_select(cand, n, p, order);
    oracle_kp *sel = (oracle_kp *)malloc(sizeof(oracle_kp) * (size_t)(N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) sel[i] = cand[order[i]];
    int total = describe_points(levels, W, H, p, sel, N, kp_out, desc_out, cap);
    free(sel);
    free(order);
    free(cand);
    free(levels);
    return total;
}

int oracle_extract_batch(int n, const uint8_t *const *imgs, const int *W, const int *H,
                         const int *pitch, const oracle_params *p, oracle_kp *kp_out,
                         double *desc_out, int cap, int *counts, int n_threads) {
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int b = 0; b < n; ++b)
        counts[b] = oracle_extract(imgs[b], W[b], H[b], pitch[b], p, kp_out + (size_t)b * cap,
                                   desc_out + (size_t)b * cap * 128, cap, NULL);
    (void)n_threads;
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------ S11: transform + ternary */

/* Sec. III-C: two order-8 transforms of a cell histogram h0..h7 built from
 * additions, subtractions and shifts; neighbouring cells alternate between
 * them (checkerboard on the cell grid). */
static void transform_set_a(const double *h, double *v) {
    v[0] = (h[2] - h[6]) / 2.0;
    v[1] = (h[3] - h[7]) / 2.0;
    v[2] = (h[0] - h[1]) / 2.0;
    v[3] = (h[2] - h[3]) / 2.0;
    v[4] = (h[4] - h[5]) / 2.0;
    v[5] = (h[6] - h[7]) / 2.0;
    v[6] = ((h[0] + h[4]) - (h[2] + h[6])) / 4.0;
    v[7] = ((h[0] + h[2] + h[4] + h[6]) - (h[1] + h[3] + h[5] + h[7])) / 8.0;
}

static void transform_set_b(const double *h, double *v) {
    v[0] = (h[0] - h[4]) / 2.0;
    v[1] = (h[1] - h[5]) / 2.0;
    v[2] = (h[7] - h[0]) / 2.0;
    v[3] = (h[1] - h[2]) / 2.0;
    v[4] = (h[3] - h[4]) / 2.0;
    v[5] = (h[5] - h[6]) / 2.0;
    v[6] = ((h[1] + h[5]) - (h[3] + h[7])) / 4.0;
    v[7] = ((h[0] + h[1] + h[2] + h[3]) - (h[4] + h[5] + h[6] + h[7])) / 8.0;
}

void oracle_transform(const double *d, double *v) {
    for (int cy = 0; cy < 4; ++cy)
        for (int cx = 0; cx < 4; ++cx) {
            int c = cy * 4 + cx;
            if (((cx + cy) & 1) == 0) transform_set_a(d + 8 * c, v + 8 * c);
            else transform_set_b(d + 8 * c, v + 8 * c);
        }
}

/* Sec. III-C: each transformed element is quantised to -1, 0, +1 by two
 * thresholds of its own. */
void oracle_ternary(const double *v, const double *t_lo, const double *t_hi, int8_t *q) {
    for (int j = 0; j < 128; ++j) q[j] = (int8_t)(v[j] < t_lo[j] ? -1 : (v[j] > t_hi[j] ? 1 : 0));
}
