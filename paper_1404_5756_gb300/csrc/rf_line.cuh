// rf_line.cuh -- one thread per (line, slice) recursive-filter sweeps.
//
// A "line" is one row (x pass) or one column (y pass) of one level of one
// variable.  Each thread walks its line causally then anticausally; the sea
// segments, coast boundary maps and land zeros follow the plan.  This is the
// general path: any line length, any mask, any stride.
#pragma once
#include <cstdint>

namespace rfvh {

struct LineArgs {
    const float *in;
    float *out;
    const float4 *coef;       // [L_nz][ny][nx]: beta, e, c1, c2 (FP32)
    const uint8_t *mask;      // [mask_nz][ny][nx]
    const int32_t *tail;      // [ncl][ny][nx]: boundary-map index or -1
    const double *tmap;       // [ntail][9] boundary maps (FP64)
    float *yscr;              // [nslices][ntail][3] backward start states
    int64_t nx, ny, nz, nslices, ntail;
    int mask_nz, L_nz, ncl;
    int along_x;              // 1: rows, 0: columns
    int iters;                // K (order 1)
};

// Third-order forward step in delta form (see rf_coef.cuh).
__device__ __forceinline__ void step3(float x, const float4 &c, float &p,
                                      float &d1, float &d2)
{
    float t = c.x * x;
    t = fmaf(-c.y, p, t);
    t = fmaf(-c.z, d1, t);
    t = fmaf(-c.w, d2, t);
    d2 += t;
    d1 += d2;
    p += d1;
}

// Transposed third-order step: adds the adjoint input g, returns the output
// beta * (lp + l1 + l2) and applies A^T to the costate (lp, l1, l2).
__device__ __forceinline__ float step3_t(float g, const float4 &c, float &lp,
                                         float &l1, float &l2)
{
    lp += g;
    float q = lp + l1;
    float S = q + l2;
    l2 = fmaf(-c.w, S, S);
    l1 = fmaf(-c.z, S, q);
    lp = fmaf(-c.y, S, lp);
    return c.x * S;
}

template <int ORDER, bool ADJ>
__global__ void __launch_bounds__(128) line_kernel(LineArgs a)
{
    const int64_t nlines = a.along_x ? a.ny : a.nx;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= nlines * a.nslices) return;
    const int64_t slice = gid / nlines, l = gid - slice * nlines;
    const int64_t k = slice % a.nz;
    const int64_t plane = a.nx * a.ny;
    const uint8_t *m = a.mask + (a.mask_nz > 1 ? k : 0) * plane;
    const float4 *cf = a.coef + (a.L_nz > 1 ? k : 0) * plane;
    const int32_t *ti = a.tail + (a.ncl > 1 ? k : 0) * plane;
    const float *src0 = a.in + slice * plane;
    float *out = a.out + slice * plane;
    float *scr = a.yscr + slice * a.ntail * 3;
    const int64_t n = a.along_x ? a.nx : a.ny;
    const int64_t base = a.along_x ? l * a.nx : l;
    const int64_t ps = a.along_x ? 1 : a.nx;
    const int K = ORDER == 3 ? 1 : a.iters;

    for (int it = 0; it < K; ++it) {
        const float *src = it == 0 ? src0 : out;
        // ---- causal sweep
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int64_t t = 0; t < n; ++t) {
            const int64_t o = base + t * ps;
            if (!m[o]) {
                s0 = s1 = s2 = 0.f;
                out[o] = 0.f;
                continue;
            }
            const float4 c = cf[o];
            const float x = src[o];
            float y;
            if (ORDER == 3) {
                if (ADJ) {
                    y = step3_t(x, c, s0, s1, s2);
                } else {
                    step3(x, c, s0, s1, s2);
                    y = s0;
                }
            } else {
                if (ADJ) {
                    s0 += x;
                    y = c.x * s0;
                    s0 = fmaf(-c.y, s0, s0);
                } else {
                    s0 += fmaf(-c.y, s0, c.x * x);
                    y = s0;
                }
            }
            out[o] = y;
            const bool end = (t == n - 1) || !m[o + ps];
            if (end) {
                const int idx = ti[o];
                if (idx >= 0) {
                    const double *M = a.tmap + (int64_t)idx * 9;
                    float *Y = scr + (int64_t)idx * 3;
                    if (ORDER == 3) {
                        const double X0 = s0, X1 = s1, X2 = s2;
                        for (int r = 0; r < 3; ++r) {
                            // forward: Y = M X; adjoint: Y = M^T X
                            double v = ADJ ? M[r] * X0 + M[3 + r] * X1 + M[6 + r] * X2
                                           : M[3 * r] * X0 + M[3 * r + 1] * X1 + M[3 * r + 2] * X2;
                            Y[r] = (float)v;
                        }
                    } else {
                        Y[0] = (float)(M[0] * (double)s0);
                    }
                }
                s0 = s1 = s2 = 0.f;
            }
        }
        // ---- anticausal sweep
        s0 = s1 = s2 = 0.f;
        for (int64_t t = n - 1; t >= 0; --t) {
            const int64_t o = base + t * ps;
            if (!m[o]) {
                s0 = s1 = s2 = 0.f;
                continue;
            }
            const bool end = (t == n - 1) || !m[o + ps];
            if (end) {
                const int idx = ti[o];
                if (idx >= 0) {
                    const float *Y = scr + (int64_t)idx * 3;
                    s0 = Y[0];
                    if (ORDER == 3) {
                        s1 = Y[1];
                        s2 = Y[2];
                    }
                } else {
                    s0 = s1 = s2 = 0.f;
                }
            }
            const float4 c = cf[o];
            const float x = out[o];
            float y;
            if (ORDER == 3) {
                if (ADJ) {
                    y = step3_t(x, c, s0, s1, s2);
                } else {
                    step3(x, c, s0, s1, s2);
                    y = s0;
                }
            } else {
                if (ADJ) {
                    s0 += x;
                    y = c.x * s0;
                    s0 = fmaf(-c.y, s0, s0);
                } else {
                    s0 += fmaf(-c.y, s0, c.x * x);
                    y = s0;
                }
            }
            out[o] = y;
        }
    }
}

}  // namespace rfvh
