/*
 * rf_oracle.c -- plain FP64 CPU oracle of the recursive-filter horizontal
 * covariance operator V_H = G_y G_x of Farina et al., "A Revised Scheme to
 * Compute Horizontal Covariances in an Oceanographic 3D-VAR Assimilation
 * System" (Sec. 2.2, Sec. 3, Appendix A).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * library; both sides were written separately from the paper.
 *
 * What it computes, step by step in the paper's notation (direct form, IEEE
 * double, built with -ffp-contract=off so no FMA contraction happens):
 *
 *  - 3rd-RF coefficients, Theorem 3.1: a_{i,0..3} from sigma_i = R_i/dx_i,
 *    alpha_{i,j} = a_{i,j}/a_{i,0}, beta_i = (2 pi sigma_i^2)^(1/4)
 *    (1 - sum_j alpha_{i,j}).
 *  - Optional q-corrected 3rd-RF (not in the paper): the a_{i,j} are taken at
 *    q_i instead of sigma_i, q_i the positive root of the impulse-response
 *    variance of Theorem 3.1's filter, 2[(P1/P0) q + ((P1/P0)^2 - 2 P2/P0) q^2],
 *    set equal to sigma_i^2, so the filter's variance is sigma_i^2; beta keeps
 *    the normalisation of sigma_i.
 *  - 1st-RF coefficients, Sec. 3.1 (Hayden relation, Eq. "crucial"):
 *    E = K dx^2/R^2, alpha = 1 + E - sqrt(E(E+2)), beta = 1 - alpha, times
 *    the Gaussian-peak factor (2 pi sigma^2)^(1/(4K)) per pass unless the
 *    unit-sum normalisation is asked for.
 *  - One line: the forward (causal) recursion then the backward
 *    (anticausal) recursion of Eqs. "fort"/"bact" (K times for the 1st-RF),
 *    with the heuristic initial conditions of Sec. 3.1 (zero state before the
 *    first point), the backward sweep run down to i = 1.
 *  - Coasts (Sec. 1 and Sec. 4: "imaginary sea points"): every maximal run of
 *    sea points of a line is a segment; it is extended on each side by
 *    n_img = ceil(img_factor * sigma_coast) imaginary points carrying input
 *    zero and the coastal point's coefficients; the recursions run over the
 *    extended segment and only the sea points are read back.  Land output 0.
 *    For K > 1 every iteration re-extends with zeros (imaginary values are not
 *    carried between iterations; carried coasts below are the option).  img_factor = +infinity is the infinite
 *    imaginary sea, realised by an extension long enough that the neglected
 *    tail is below FP64 resolution (n_imaginary).
 *  - Constant-extension coasts (an option; one of the alternative coast
 *    conditions the Conclusions leave for future work): the imaginary
 *    points carry the value of the adjacent sea point (the first sea point's
 *    value on the left, the last one's on the right) instead of zero.  The
 *    extension E_c is then no longer a zero padding, and its transpose adds
 *    the adjoint's values at the imaginary points to the edge point they
 *    copied.
 *  - Carried coasts (an option; another of those alternative conditions):
 *    for the 1st-RF with K > 1 iterations the segment is extended once with
 *    zero-input imaginary points and all K iterations run over the extended
 *    segment, so the values the imaginary points take in one iteration feed
 *    the next; only the final result is read back: R G_ext^K R^T instead of
 *    (R G_ext R^T)^K.  The adjoint is R (G_ext^T)^K R^T.  With K = 1 (and for
 *    the 3rd-RF) it is the zero-input coast.
 *  - The 2-D operator V_H = G_y G_x (Sec. 2.2): rows (x) first, then columns
 *    (y), on every level of every variable.
 *  - The adjoint V_H^T = G_x^T G_y^T, written out as the transposed
 *    triangular solves of each pass (the gradient of the 3D-VAR cost, Eq.
 *    "eight", needs it; the paper does not write it down).
 *
 * Pins (tests/test_oracle_pins.py): dense triangular-solve matrices on tiny
 * lines, the closed-form DC gain sqrt(2 pi) sigma, the closed-form impulse
 * variance of the 3rd-RF and Hayden's sigma^2 for the 1st-RF, the
 * Abramowitz-Stegun factorisation behind the constants, land isolation,
 * constant-field preservation and the adjoint dot-product test.
 * The coastal mechanism itself has no printed data: its exact behaviour
 * against OceanVar is parity unpinned (only its internal consistency with a
 * padded line is pinned).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

/* The q of the q-corrected 3rd-RF: variance(q) = A q^2 + B q = sigma^2 with
 * A = 2 ((P1/P0)^2 - 2 P2/P0), B = 2 P1/P0, solved as 2 sigma^2 / (B + root)
 * (no cancellation at small sigma). */
double orc_q_of_sigma(double sigma)
{
    double r1 = 5.788982 / 3.738128, r2 = 3.382473 / 3.738128;
    double A = 2.0 * (r1 * r1 - 2.0 * r2), B = 2.0 * r1;
    double s2 = sigma * sigma;
    return 2.0 * s2 / (B + sqrt(B * B + 4.0 * A * s2));
}

/* Theorem 3.1: a_{i,0..3}, alpha_{i,1..3} and beta_i for one grid point
 * (qcorr: the a_{i,j} at q(sigma), beta still normalised with sigma). */
void orc_rf3_coeffs(double sigma, int norm, int qcorr, double a[4], double alpha[3],
                    double *beta)
{
    double s = qcorr ? orc_q_of_sigma(sigma) : sigma, s2 = s * s, s3 = s2 * s;
    a[0] = 3.738128 + 5.788982 * s + 3.382473 * s2 + 1.000000 * s3;
    a[1] = 5.788982 * s + 6.764946 * s2 + 3.000000 * s3;
    a[2] = -3.382473 * s2 - 3.000000 * s3;
    a[3] = 1.000000 * s3;
    alpha[0] = a[1] / a[0];
    alpha[1] = a[2] / a[0];
    alpha[2] = a[3] / a[0];
    double g = (norm == 1) ? 1.0 : pow(2.0 * ORC_PI * sigma * sigma, 0.25);
    *beta = g * (1.0 - (alpha[0] + alpha[1] + alpha[2]));
}

/* Sec. 3.1, first-order filter iterated K times (Hayden relation). */
void orc_rf1_coeffs(double sigma, int K, int norm, double *alpha,
                    double *beta)
{
    double E = (double)K / (sigma * sigma);   /* K dx^2 / R^2 */
    double r = sqrt(E * (E + 2.0));
    *alpha = 1.0 + E - r;
    double g = (norm == 1) ? 1.0 : pow(2.0 * ORC_PI * sigma * sigma,
                                       1.0 / (4.0 * (double)K));
    *beta = (-E + r) * g;
}

/* Workspace for one extended segment. */
typedef struct {
    int64_t cap;
    double *alpha;  /* [cap][3] */
    double *beta;   /* [cap]    */
    double *x;      /* [cap]    */
    double *y;      /* [cap]    */
} orc_ws;

static int ws_reserve(orc_ws *w, int64_t m)
{
    if (m <= w->cap) return ORC_OK;
    free(w->alpha); free(w->beta); free(w->x); free(w->y);
    w->alpha = (double *)malloc(sizeof(double) * 3 * (size_t)m);
    w->beta = (double *)malloc(sizeof(double) * (size_t)m);
    w->x = (double *)malloc(sizeof(double) * (size_t)m);
    w->y = (double *)malloc(sizeof(double) * (size_t)m);
    if (!w->alpha || !w->beta || !w->x || !w->y) { w->cap = 0; return ORC_ENOMEM; }
    w->cap = m;
    return ORC_OK;
}

static void ws_free(orc_ws *w)
{
    free(w->alpha); free(w->beta); free(w->x); free(w->y);
    memset(w, 0, sizeof(*w));
}

/* Imaginary points at a coast whose sea point has length scale sigma_coast.
 * img_factor = +infinity is the infinite imaginary sea: the recursions run on
 * forever with zero input, and since the filters' poles lie inside the unit
 * circle (|z| <= 1 - 0.5/(1 + sigma) for both filters; the pins check the
 * spectral radius) the extension is cut at ceil(60 (1 + 2 sigma_coast))
 * points, beyond which the neglected part of the response is below e^-100 of
 * it, far under FP64 resolution. */
static int64_t n_imaginary(double img_factor, double sigma_coast)
{
    if (!(img_factor > 0.0)) return 0;
    if (isinf(img_factor)) return (int64_t)ceil(60.0 * (1.0 + 2.0 * sigma_coast));
    return (int64_t)ceil(img_factor * sigma_coast);
}

/* Public: the number of imaginary points the oracle uses at a coast. */
int64_t orc_n_imaginary(double img_factor, double sigma_coast)
{
    return n_imaginary(img_factor, sigma_coast);
}

/* Coefficients of the extended segment: imaginary points take the
 * coefficients of the adjacent coastal sea point. */
static void fill_coeffs(int order, int K, int norm, int qcorr, const double *sig,
                        int64_t L, int64_t nl, int64_t nr, orc_ws *w)
{
    int64_t m = nl + L + nr;
    for (int64_t r = 0; r < m; ++r) {
        int64_t src = r < nl ? 0 : (r >= nl + L ? L - 1 : r - nl);
        double *al = w->alpha + 3 * r;
        if (order == 3) {
            double a[4];
            orc_rf3_coeffs(sig[src], norm, qcorr, a, al, &w->beta[r]);
        } else {
            orc_rf1_coeffs(sig[src], K, norm, &al[0], &w->beta[r]);
            al[1] = 0.0;
            al[2] = 0.0;
        }
    }
}

/* Forward recursion (Eq. "fort") then backward recursion (Eq. "bact") over
 * the extended segment x[0..m) with zero state outside it; result in x. */
static void forward_backward(int64_t m, const double *alpha, const double *beta,
                             double *x, double *p)
{
    for (int64_t i = 0; i < m; ++i) {
        double v = beta[i] * x[i];
        for (int j = 1; j <= 3; ++j)
            if (i - j >= 0) v += alpha[3 * i + j - 1] * p[i - j];
        p[i] = v;
    }
    for (int64_t i = m - 1; i >= 0; --i) {
        double v = beta[i] * p[i];
        for (int j = 1; j <= 3; ++j)
            if (i + j < m) v += alpha[3 * i + j - 1] * x[i + j];
        x[i] = v;
    }
}

/* Transpose of forward_backward: G = U^-1 D L^-1 D, so
 * G^T = D L^-T D U^-T.  U^T z = y is solved causally with the coefficients
 * of the earlier point (alpha_{r-j,j}); L^T w = v anticausally with the
 * coefficients of the later point (alpha_{r+j,j}). */
static void forward_backward_adjoint(int64_t m, const double *alpha,
                                     const double *beta, double *x, double *z)
{
    for (int64_t r = 0; r < m; ++r) {
        double v = x[r];
        for (int j = 1; j <= 3; ++j)
            if (r - j >= 0) v += alpha[3 * (r - j) + j - 1] * z[r - j];
        z[r] = v;
    }
    for (int64_t r = 0; r < m; ++r) z[r] *= beta[r];
    for (int64_t r = m - 1; r >= 0; --r) {
        double v = z[r];
        for (int j = 1; j <= 3; ++j)
            if (r + j < m) v += alpha[3 * (r + j) + j - 1] * x[r + j];
        x[r] = v;
    }
    for (int64_t r = 0; r < m; ++r) x[r] *= beta[r];
}

/* One line of n points.  mask[i] != 0 marks sea.  sig[i] = R_i/dx_i.
 * coast: 0 imaginary points carry zero, 1 they carry the adjacent sea value,
 * 2 they start at zero and keep their values from iteration to iteration. */
static int line_apply(int order, int iters, int adjoint, double img_factor,
                      int norm, int qcorr, int coast, int64_t n, const uint8_t *mask,
                      const double *sig, const double *in, double *out,
                      orc_ws *w)
{
    int64_t i = 0;
    while (i < n) {
        if (!mask[i]) { out[i] = 0.0; ++i; continue; }
        int64_t b = i;
        while (i < n && mask[i]) ++i;
        int64_t L = i - b;
        for (int64_t t = b; t < i; ++t)
            if (!(sig[t] > 0.0) || !isfinite(sig[t])) return ORC_EINVAL;
        int64_t nl = n_imaginary(img_factor, sig[b]);
        int64_t nr = n_imaginary(img_factor, sig[i - 1]);
        int64_t m = nl + L + nr;
        if (ws_reserve(w, m) != ORC_OK) return ORC_ENOMEM;
        fill_coeffs(order, iters, norm, qcorr, sig + b, L, nl, nr, w);
        for (int64_t t = 0; t < L; ++t) out[b + t] = in[b + t];
        for (int k = 0; k < iters; ++k) {
            /* extend (E, or R^T for the adjoint): zeros, or for the forward
             * constant extension the edge values; carried coasts extend
             * before the first iteration only */
            if (coast != 2 || k == 0) {
                for (int64_t r = 0; r < m; ++r) w->x[r] = 0.0;
                for (int64_t t = 0; t < L; ++t) w->x[nl + t] = out[b + t];
            }
            if (coast == 1 && !adjoint) {
                for (int64_t r = 0; r < nl; ++r) w->x[r] = out[b];
                for (int64_t r = nl + L; r < m; ++r) w->x[r] = out[b + L - 1];
            }
            if (adjoint)
                forward_backward_adjoint(m, w->alpha, w->beta, w->x, w->y);
            else
                forward_backward(m, w->alpha, w->beta, w->x, w->y);
            /* restrict to the sea points (R, or E^T for the adjoint: with
             * constant extension the imaginary values go to the edge point
             * they copied); carried coasts keep the extended segment */
            if (coast == 2 && k < iters - 1) continue;
            for (int64_t t = 0; t < L; ++t) out[b + t] = w->x[nl + t];
            if (coast == 1 && adjoint) {
                for (int64_t r = 0; r < nl; ++r) out[b] += w->x[r];
                for (int64_t r = nl + L; r < m; ++r) out[b + L - 1] += w->x[r];
            }
        }
    }
    return ORC_OK;
}

static int check_opts(int order, int iters, int qcorr, int coast)
{
    if (order != 1 && order != 3) return ORC_EINVAL;
    if (coast < 0 || coast > 2) return ORC_EINVAL;
    if (qcorr && order != 3) return ORC_EINVAL;
    if (iters < 1) return ORC_EINVAL;
    if (order == 3 && iters != 1) return ORC_EINVAL;
    return ORC_OK;
}

/* Public: one 1-D line (the operator G of one direction). */
int orc_line(int order, int iters, int adjoint, double img_factor, int norm,
             int qcorr, int coast, int64_t n, const uint8_t *mask, const double *sig,
             const double *in, double *out)
{
    if (check_opts(order, iters, qcorr, coast) != ORC_OK || n < 0) return ORC_EINVAL;
    orc_ws w = {0};
    int rc = line_apply(order, iters, adjoint, img_factor, norm, qcorr, coast, n, mask, sig,
                        in, out, &w);
    ws_free(&w);
    return rc;
}

/* One level slice of one variable: V_H (or its adjoint) of src into dst,
 * with the slice's mask and length scales; tmp is a plane of scratch and
 * li/lo/ls/lm line buffers of max(nx, ny). */
static int slice_apply(int order, int iters, int adjoint, double img_factor, int norm,
                       int qcorr, int coast, int64_t nx, int64_t ny, const uint8_t *mk,
                       const double *sx, const double *sy, const double *src, double *dst,
                       double *tmp, double *li, double *lo, double *ls, uint8_t *lm,
                       orc_ws *w)
{
    int rc = ORC_OK;
    for (int pass = 0; pass < 2 && rc == ORC_OK; ++pass) {
        /* forward: x then y; adjoint: y then x */
        int along_x = adjoint ? (pass == 1) : (pass == 0);
        const double *a = pass == 0 ? src : tmp;
        double *b = pass == 0 ? tmp : dst;
        if (along_x) {
            for (int64_t j = 0; j < ny && rc == ORC_OK; ++j)
                rc = line_apply(order, iters, adjoint, img_factor, norm, qcorr, coast,
                                nx, mk + j * nx, sx + j * nx, a + j * nx, b + j * nx, w);
        } else {
            for (int64_t i = 0; i < nx && rc == ORC_OK; ++i) {
                for (int64_t j = 0; j < ny; ++j) {
                    lm[j] = mk[j * nx + i];
                    ls[j] = sy[j * nx + i];
                    li[j] = a[j * nx + i];
                }
                rc = line_apply(order, iters, adjoint, img_factor, norm, qcorr, coast,
                                ny, lm, ls, li, lo, w);
                for (int64_t j = 0; j < ny; ++j) b[j * nx + i] = lo[j];
            }
        }
    }
    return rc;
}

/* Threads of orc_vh's loop over the (variable, level) slices, the paper's
 * own parallel axis (OpenMP over levels, Sec. 5); 1 by default.  The slices
 * are independent and each is computed sequentially, so the result does not
 * depend on the thread count. */
static int g_threads = 1;

int orc_set_threads(int n)
{
    g_threads = n < 1 ? 1 : n;
    return g_threads;
}

/* Public: V_H = G_y G_x (or its adjoint G_x^T G_y^T) on fields laid out
 * [nvar][nz][ny][nx], x fastest.  mask is [mask_nz][ny][nx], Lx and Ly are
 * [L_nz][ny][nx] in grid units; mask_nz and L_nz are 1 (shared by every
 * level) or nz.  in and out may not alias. */
int orc_vh(int order, int iters, int adjoint, double img_factor, int norm,
           int qcorr, int coast, int64_t nx, int64_t ny, int64_t nz, int64_t nvar,
           const uint8_t *mask, int64_t mask_nz, const double *Lx,
           const double *Ly, int64_t L_nz, const double *in, double *out)
{
    if (check_opts(order, iters, qcorr, coast) != ORC_OK) return ORC_EINVAL;
    if (nx < 0 || ny < 0 || nz < 0 || nvar < 0) return ORC_EINVAL;
    if (!(mask_nz == 1 || mask_nz == nz) || !(L_nz == 1 || L_nz == nz))
        return ORC_EINVAL;
    const int64_t plane = nx * ny, nmax = nx > ny ? nx : ny, nslices = nvar * nz;
    int rc = ORC_OK;
#pragma omp parallel num_threads(g_threads) if (g_threads > 1)
    {
        double *tmp = (double *)malloc(sizeof(double) * (size_t)(plane ? plane : 1));
        double *li = (double *)malloc(sizeof(double) * (size_t)(nmax ? nmax : 1));
        double *lo = (double *)malloc(sizeof(double) * (size_t)(nmax ? nmax : 1));
        double *ls = (double *)malloc(sizeof(double) * (size_t)(nmax ? nmax : 1));
        uint8_t *lm = (uint8_t *)malloc((size_t)(nmax ? nmax : 1));
        orc_ws w = {0};
        int my = (tmp && li && lo && ls && lm) ? ORC_OK : ORC_ENOMEM;
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < nslices; ++s) {
            if (my != ORC_OK) continue;
            const int64_t v = s / nz, k = s % nz;
            (void)v;
            my = slice_apply(order, iters, adjoint, img_factor, norm, qcorr, coast, nx, ny,
                             mask + (mask_nz == 1 ? 0 : k) * plane,
                             Lx + (L_nz == 1 ? 0 : k) * plane, Ly + (L_nz == 1 ? 0 : k) * plane,
                             in + s * plane, out + s * plane, tmp, li, lo, ls, lm, &w);
        }
        if (my != ORC_OK) {
#pragma omp critical
            rc = my;
        }
        ws_free(&w);
        free(tmp); free(li); free(lo); free(ls); free(lm);
    }
    return rc;
}
