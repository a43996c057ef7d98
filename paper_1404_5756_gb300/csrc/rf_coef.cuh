// rf_coef.cuh -- FP64 filter coefficients and coastal boundary maps.
//
// Third-order filter (Theorem 3.1): with sigma = R/dx,
//   a0 = P0 + P1 s + P2 s^2 + s^3,  alpha_j = a_j/a0,
//   beta = (2 pi s^2)^(1/4) (1 - sum_j alpha_j) = (2 pi s^2)^(1/4) P0/a0,
// because a0 - a1 - a2 - a3 = P0 exactly for the Theorem's a_j.  The GPU runs
// the same recursion in its delta (difference) realisation: with
//   d1_i = p_i - p_{i-1},  d2_i = d1_i - d1_{i-1},
// writing a_{i,0} p_i - sum_j a_{i,j} p_{i-j} as a polynomial in the backward
// difference (Appendix A, s = 1 - z^-1) gives, per point,
//   t   = beta s_i - e p_{i-1} - c1 d1_{i-1} - c2 d2_{i-1}
//   d2_i = d2_{i-1} + t,  d1_i = d1_{i-1} + d2_i,  p_i = p_{i-1} + d1_i
// with e = P0/a0, c1 = (P0 + P1 s)/a0, c2 = (P0 + P1 s + P2 s^2)/a0.  This is
// an exact identity with the direct form, even with per-point coefficients,
// and keeps FP32 rounding small when 1 - sum alpha is tiny (large sigma).
// First-order filter (Sec. 3.1, Hayden): E = K/sigma^2, e = 1 - alpha =
// sqrt(E(E+2)) - E, and the step is p_i = p_{i-1} + (beta s_i - e p_{i-1}).
//
// q-corrected third-order filter (an option, not the paper's filter): the
// impulse response of the Theorem 3.1 filter at scale s has variance
// 2 (P1/P0) s + 2 ((P1/P0)^2 - 2 P2/P0) s^2 (the first two cumulants of
// 1/D(s(1 - e^t)), D the cubic of Appendix A), not s^2.  Taking the a_j at the
// positive root q of variance(q) = sigma^2 gives variance sigma^2; beta keeps
// the normalisation of sigma, so the DC gain stays sqrt(2 pi) sigma.
#pragma once
#include <cstdint>

namespace rfvh {

// Theorem 3.1 constants, as printed.
constexpr double kP0 = 3.738128;
constexpr double kP1 = 5.788982;
constexpr double kP2 = 3.382473;
constexpr double kTwoPi = 6.283185307179586476925286766559;

struct Coef64 {
    double beta, e, c1, c2;
};

// Scale q with variance(q) = sigma^2, as 2 sigma^2 / (B + sqrt(B^2 + 4 A
// sigma^2)) for A q^2 + B q = sigma^2 (no cancellation at small sigma).
__host__ __device__ inline double q_corrected(double sigma)
{
    const double r1 = kP1 / kP0, r2 = kP2 / kP0;
    const double A = 2.0 * (r1 * r1 - 2.0 * r2), Bq = 2.0 * r1;
    const double s2 = sigma * sigma;
    return 2.0 * s2 / (Bq + sqrt(Bq * Bq + 4.0 * A * s2));
}

// Per-point coefficients in FP64 (sigma > 0, finite).  norm: 0 Gaussian peak,
// 1 unit sum.  qc: q-corrected third-order filter.  For order 1, c1 = c2 = 0.
__host__ __device__ inline Coef64 coef_fp64(double sigma, int order, int K,
                                            int norm, bool qc = false)
{
    Coef64 c;
    if (order == 3) {
        double s = qc ? q_corrected(sigma) : sigma;
        double a0 = kP0 + s * (kP1 + s * (kP2 + s));
        double inv = 1.0 / a0;
        c.e = kP0 * inv;
        c.c1 = (kP0 + kP1 * s) * inv;
        c.c2 = (kP0 + s * (kP1 + kP2 * s)) * inv;
        double g = norm == 1 ? 1.0 : sqrt(sqrt(kTwoPi) * sigma);
        c.beta = g * c.e;
    } else {
        double E = (double)K / (sigma * sigma);
        double r = sqrt(E * (E + 2.0));
        c.e = 2.0 * E / (r + E);      // = r - E without cancellation
        c.c1 = 0.0;
        c.c2 = 0.0;
        double g = norm == 1 ? 1.0 : pow(kTwoPi * sigma * sigma, 1.0 / (4.0 * K));
        c.beta = g * c.e;
    }
    return c;
}

// Boundary map of one coast end.  Running the forward recursion from the
// state X at the last sea point through n imaginary points (zero input, the
// coastal coefficients), then the backward recursion from zero state at the
// far end back to the coast, leaves the backward state Y = M X at the first
// imaginary point, with (delta basis, A the one-step matrix, b the input
// column, c = (1,0,0) the output row)
//   M = sum_{k=1..n} A^{k-1} b c^T A^k.
// Order 3 writes the 3x3 M row-major into m[0..9); order 1 writes m[0].
__host__ __device__ inline void tail_map_fp64(double sigma, int n_img, int order,
                                              int K, int norm, bool qc, double *m)
{
    Coef64 c = coef_fp64(sigma, order, K, norm, qc);
    if (order == 1) {
        double a = 1.0 - c.e, acc = 0.0, v = c.beta, w = a;
        for (int k = 1; k <= n_img; ++k) {
            acc += v * w;
            v *= a;
            w *= a;
        }
        m[0] = acc;
        for (int r = 1; r < 9; ++r) m[r] = 0.0;
        return;
    }
    // one-step matrix acting on (p, d1, d2)
    const double A[9] = {1.0 - c.e, 1.0 - c.c1, 1.0 - c.c2,
                         -c.e,      1.0 - c.c1, 1.0 - c.c2,
                         -c.e,      -c.c1,      1.0 - c.c2};
    double v[3] = {c.beta, c.beta, c.beta};    // A^{k-1} b
    double w[3] = {A[0], A[1], A[2]};          // c^T A^k (first row of A^k)
    for (int r = 0; r < 9; ++r) m[r] = 0.0;
    for (int k = 1; k <= n_img; ++k) {
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) m[3 * r + q] += v[r] * w[q];
        double nv[3], nw[3];
        for (int r = 0; r < 3; ++r) {
            nv[r] = A[3 * r] * v[0] + A[3 * r + 1] * v[1] + A[3 * r + 2] * v[2];
            nw[r] = w[0] * A[r] + w[1] * A[3 + r] + w[2] * A[6 + r];
        }
        for (int r = 0; r < 3; ++r) {
            v[r] = nv[r];
            w[r] = nw[r];
        }
    }
}

// Boundary map of the infinite imaginary sea (img_factor = infinity): the
// limit of tail_map_fp64 as n -> infinity,
//   M = sum_{j>=0} A^j Q A^j,  Q = b c^T A,
// which converges because the filter's poles lie inside the unit circle and
// is the solution of the Stein equation M = Q + A M A.  Solved directly as
// the 9 x 9 linear system (I - K) vec(M) = vec(Q), K[(r,q),(s,t)] =
// A[r][s] A[t][q] (row-major vec), by Gaussian elimination with partial
// pivoting in FP64.  Order 1: M = b a / (1 - a^2) with a = 1 - e.
__host__ __device__ inline void tail_map_inf_fp64(double sigma, int order, int K, int norm,
                                                  bool qc, double *m)
{
    Coef64 c = coef_fp64(sigma, order, K, norm, qc);
    for (int r = 0; r < 9; ++r) m[r] = 0.0;
    if (order == 1) {
        const double a = 1.0 - c.e;
        m[0] = c.beta * a / ((1.0 - a) * (1.0 + a));
        return;
    }
    const double A[9] = {1.0 - c.e, 1.0 - c.c1, 1.0 - c.c2,
                         -c.e,      1.0 - c.c1, 1.0 - c.c2,
                         -c.e,      -c.c1,      1.0 - c.c2};
    double S[9][10];   // [I - K | vec Q]
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            const int row = 3 * r + q;
            for (int s = 0; s < 3; ++s)
                for (int t = 0; t < 3; ++t)
                    S[row][3 * s + t] = (row == 3 * s + t ? 1.0 : 0.0) - A[3 * r + s] * A[3 * t + q];
            S[row][9] = c.beta * A[q];   // Q = b c^T A, b = beta (1,1,1), c^T A = row 0 of A
        }
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(S[r][col]) > fabs(S[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k < 10; ++k) {
                const double t = S[col][k];
                S[col][k] = S[piv][k];
                S[piv][k] = t;
            }
        for (int r = col + 1; r < 9; ++r) {
            const double f = S[r][col] / S[col][col];
            for (int k = col; k < 10; ++k) S[r][k] -= f * S[col][k];
        }
    }
    for (int r = 8; r >= 0; --r) {
        double v = S[r][9];
        for (int k = r + 1; k < 9; ++k) v -= S[r][k] * m[k];
        m[r] = v / S[r][r];
    }
}

// History weights of the carried coasts (an option, 1st-RF with K > 1
// iterations): the imaginary points of a segment start at zero and keep the
// values each iteration leaves in them, so after iteration k they hold a
// linear function of the boundary states the sea saw in iterations 1..k.
// With a = 1 - e and beta the coastal point's coefficients:
//   right end (n points after the last sea point): X is the state the first
//     sweep leaves at the last sea point, u the points' content; one iteration
//     maps (X, u) to the second sweep's start state Y and the new content u';
//   left end (n points before the first sea point): v the content; the first
//     sweep enters the sea with state H(v); S is the state the second sweep
//     leaves at the first sea point; one iteration maps (S, v) to v'.
// Forward (G = anticausal o causal, both stepping p = a p + beta x):
//   right: p = X, p_t = a p_{t-1} + beta u_t (t = 1..n); y_{n+1} = 0,
//          y_t = a y_{t+1} + beta p_t; Y = y_1, u' = y;
//   left:  p_{n+1} = 0, p_t = a p_{t+1} + beta v_t (t = n..1, t = 1 next to
//          the sea); H = p_1; y_0 = S, y_t = a y_{t-1} + beta p_t; v' = y.
// Adjoint (G^T: the transposed steps l = l + x, out = beta l, l = a l, first
// left to right, then right to left):
//   right: l = X; for t = 1..n: l += u_t, w_t = beta l, l = a l; m = 0; for
//          t = n..1: m += w_t, u'_t = beta m, m = a m; Y = m;
//   left:  l = 0; for t = n..1: l += v_t, w_t = beta l, l = a l; H = l;
//          m = S; for t = 1..n: m += w_t, v'_t = beta m, m = a m.
// By linearity, in iteration k (1-based) the start state injected at the
// segment's end is Y_k = M X_k + sum_{d=1..k-1} mu_d X_{k-d} and the state
// entering its first point is H_k = sum_{d=1..k-1} lambda_d S_{k-d}, with
//   mu_d = Y(0, psi_d), psi_1 = u'(1, 0), psi_{d+1} = u'(0, psi_d);
//   lambda_d = H(chi_d), chi_1 = v'(1, 0), chi_{d+1} = v'(0, chi_d).
// carry_weights_fp64 writes mu_1..mu_{K-1} or lambda_1..lambda_{K-1} of one
// end (n imaginary points at length scale sigma) into w, using buf (2n
// doubles) as scratch.
__host__ __device__ inline void carry_weights_fp64(double sigma, int64_t n, int K, int norm,
                                                   bool adjoint, bool right, double *buf,
                                                   double *w)
{
    const Coef64 c = coef_fp64(sigma, 1, K, norm);
    const double a = 1.0 - c.e, b = c.beta;
    double *z = buf, *t = buf + n;   // content, scratch
    // one iteration of the run with boundary state bs and content z (in
    // place -> z'); returns Y (right) or H (left, of the incoming content)
    auto step = [&](double bs) -> double {
        double out = 0.0;
        if (!adjoint) {
            if (right) {
                double p = bs;
                for (int64_t i = 0; i < n; ++i) t[i] = p = a * p + b * z[i];
                double y = 0.0;
                for (int64_t i = n - 1; i >= 0; --i) z[i] = y = a * y + b * t[i];
                out = n > 0 ? z[0] : 0.0;
            } else {
                double p = 0.0;
                for (int64_t i = n - 1; i >= 0; --i) t[i] = p = a * p + b * z[i];
                out = n > 0 ? t[0] : 0.0;
                double y = bs;
                for (int64_t i = 0; i < n; ++i) z[i] = y = a * y + b * t[i];
            }
        } else {
            if (right) {
                double l = bs;
                for (int64_t i = 0; i < n; ++i) {
                    l += z[i];
                    t[i] = b * l;
                    l *= a;
                }
                double m = 0.0;
                for (int64_t i = n - 1; i >= 0; --i) {
                    m += t[i];
                    z[i] = b * m;
                    m *= a;
                }
                out = m;
            } else {
                double l = 0.0;
                for (int64_t i = n - 1; i >= 0; --i) {
                    l += z[i];
                    t[i] = b * l;
                    l *= a;
                }
                out = l;
                double m = bs;
                for (int64_t i = 0; i < n; ++i) {
                    m += t[i];
                    z[i] = b * m;
                    m *= a;
                }
            }
        }
        return out;
    };
    for (int64_t i = 0; i < n; ++i) z[i] = 0.0;
    step(1.0);   // z = psi_1 (chi_1)
    for (int d = 1; d < K; ++d) {
        if (right) {
            w[d - 1] = step(0.0);   // Y(0, psi_d), z -> psi_{d+1}
        } else {
            // H(chi_d) is the incoming content's entering state; then chi_{d+1}
            w[d - 1] = step(0.0);
        }
    }
}

// Vectors of the constant-extension coasts (an option: the imaginary points
// carry the adjacent sea value instead of zero; one of the other coastal
// boundary conditions the Conclusions leave for future work).  With A, b, c
// as above and u_k = sum_{j<k} A^j b the state after k steps of unit input
// from zero:
//   head: the n imaginary points before a segment carry its first value x_a,
//         so the causal state entering the first sea point is x_a s with
//         s = u_n;
//   tail: the n imaginary points after a segment carry its last value x_e,
//         so their forward outputs gain x_e f_k, f_k = c^T u_k, and the
//         backward start state becomes M X + x_e m with
//         m = sum_{k=1..n} A^{k-1} b f_k.
// Order 3 writes 3 entries (delta basis p, d1, d2); order 1 writes v[0].
__host__ __device__ inline void coast_vectors_fp64(double sigma, int n_img, int order, int K,
                                                   int norm, bool qc, double *head, double *tail)
{
    Coef64 c = coef_fp64(sigma, order, K, norm, qc);
    for (int r = 0; r < 3; ++r) head[r] = tail[r] = 0.0;
    if (order == 1) {
        const double a = 1.0 - c.e;
        double u = 0.0, v = c.beta;        // u_k, A^{k-1} b
        for (int k = 1; k <= n_img; ++k) {
            u = a * u + c.beta;
            tail[0] += v * u;
            v *= a;
        }
        head[0] = u;
        return;
    }
    const double A[9] = {1.0 - c.e, 1.0 - c.c1, 1.0 - c.c2,
                         -c.e,      1.0 - c.c1, 1.0 - c.c2,
                         -c.e,      -c.c1,      1.0 - c.c2};
    double u[3] = {0.0, 0.0, 0.0};
    double v[3] = {c.beta, c.beta, c.beta};    // A^{k-1} b
    for (int k = 1; k <= n_img; ++k) {
        double nu[3], nv[3];
        for (int r = 0; r < 3; ++r) {
            nu[r] = A[3 * r] * u[0] + A[3 * r + 1] * u[1] + A[3 * r + 2] * u[2] + c.beta;
            nv[r] = A[3 * r] * v[0] + A[3 * r + 1] * v[1] + A[3 * r + 2] * v[2];
        }
        for (int r = 0; r < 3; ++r) {
            u[r] = nu[r];
            tail[r] += v[r] * u[0];
        }
        for (int r = 0; r < 3; ++r) v[r] = nv[r];
    }
    for (int r = 0; r < 3; ++r) head[r] = u[r];
}

}  // namespace rfvh
