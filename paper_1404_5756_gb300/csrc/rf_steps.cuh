// rf_steps.cuh -- one grid point of the recursive filters, forward and
// transposed, in the delta realisation (see rf_coef.cuh for the identity
// with Theorem 3.1's direct form).
//
// Per point the plan stores c = (beta, e, c1, c2) in FP32.  Land points
// carry c = (0, 0, 0, 1) and the reset factor g = 0 (g = 1 at sea); with
// those values one step maps any state to exactly zero and outputs zero, so
// land needs no branch.  The sign bit of c2 marks the last sea point of a
// segment (the "right end" where the coastal boundary map applies); callers
// strip it with fabsf before stepping.
//
// Forward step (third order), state (p, d1, d2) = (p_i, p_i - p_{i-1},
// second difference), input x:
//   t  = beta x - c2 d2 - c1 d1 - e p
//   d2 = d2 + t;  d1 = g d1 + d2;  p = g p + d1;   output p
// With g = 1 this is A_i X + b_i x, A_i the one-step matrix of rf_coef.cuh.
//
// Transposed step (third order), costate (lp, l1, l2) of (p, d1, d2), input
// y (zeroed at land by the caller): the exact transpose of the forward step
// written as the reversed sequence of its elementary operations,
//   lp = g lp + y;  l1 = g l1 + lp;  l2 = g l2 + l1;  output beta l2
//   lp -= e l2;  l1 -= c1 l2;  l2 -= c2 l2
// which equals A_i^T acting on the costate after adding y, with output
// beta (lp + l1 + l2).
#pragma once

namespace rfvh {

__device__ __forceinline__ float reset_factor(const float4 &c)
{
    return c.x != 0.f ? 1.f : 0.f;
}

__device__ __forceinline__ bool right_end(const float4 &c)
{
    return __float_as_uint(c.w) >> 31;
}

__device__ __forceinline__ float fwd3(float x, const float4 &c, float g, float &p,
                                      float &d1, float &d2)
{
    float t = c.x * x;
    t = fmaf(-c.w, d2, t);
    t = fmaf(-c.z, d1, t);
    t = fmaf(-c.y, p, t);
    d2 += t;
    d1 = fmaf(g, d1, d2);
    p = fmaf(g, p, d1);
    return p;
}

__device__ __forceinline__ float adj3(float y, const float4 &c, float g, float &lp,
                                      float &l1, float &l2)
{
    lp = fmaf(g, lp, y);
    l1 = fmaf(g, l1, lp);
    l2 = fmaf(g, l2, l1);
    const float out = c.x * l2;
    lp = fmaf(-c.y, l2, lp);
    l1 = fmaf(-c.z, l2, l1);
    l2 = fmaf(-c.w, l2, l2);
    return out;
}

// First order (Sec. 3.1), state p: t = beta x - e p;  p = g p + t.
__device__ __forceinline__ float fwd1(float x, const float4 &c, float g, float &p)
{
    const float t = fmaf(-c.y, p, c.x * x);
    p = fmaf(g, p, t);
    return p;
}

// Transposed first order: lp = g lp + y; output beta lp; lp -= e lp.
__device__ __forceinline__ float adj1(float y, const float4 &c, float g, float &lp)
{
    lp = fmaf(g, lp, y);
    const float out = c.x * lp;
    lp = fmaf(-c.y, lp, lp);
    return out;
}

// One step of the sweep kind selected at compile time.  s[0..2] is the
// (co)state; for order 1 only s[0] is used.  c must have c.w >= 0.
template <int ORDER, bool ADJ>
__device__ __forceinline__ float step(float x, const float4 &c, float g, float *s)
{
    if (ORDER == 3) {
        return ADJ ? adj3(x, c, g, s[0], s[1], s[2]) : fwd3(x, c, g, s[0], s[1], s[2]);
    } else {
        return ADJ ? adj1(x, c, g, s[0]) : fwd1(x, c, g, s[0]);
    }
}

// Coastal boundary map: forward Y = M X, adjoint Y = M^T X, in FP64.
template <int ORDER, bool ADJ>
__device__ __forceinline__ void apply_tail(const double *M, const float *X, float *Y)
{
    if (ORDER == 3) {
        const double x0 = X[0], x1 = X[1], x2 = X[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const double v = ADJ ? M[r] * x0 + M[3 + r] * x1 + M[6 + r] * x2
                                 : M[3 * r] * x0 + M[3 * r + 1] * x1 + M[3 * r + 2] * x2;
            Y[r] = (float)v;
        }
    } else {
        Y[0] = (float)(M[0] * (double)X[0]);
    }
}

}  // namespace rfvh
