// rf_steps.cuh -- one grid point of the recursive filters, forward and
// transposed, in the delta realisation (see rf_coef.cuh for the identity
// with Theorem 3.1's direct form).
//
// Per point the plan stores c = (beta, -e, -c1, -c2) in FP32 (the negated
// coefficients feed fused multiply-adds directly).  Land points carry
// c = (0, 0, 0, -1) and the reset factor g = 0 (g = 1 at sea); with those
// values one step maps any state to exactly zero and outputs zero, so land
// needs no branch.  In the plan's line-major copy the sign bit of beta marks
// the last sea point of a segment (the "right end" where the coastal
// boundary map applies); kernels strip it with fabsf before stepping.
//
// Forward step (third order), state (p, d1, d2) = (p_i, p_i - p_{i-1},
// second difference), input x:
//   t  = beta x - c2 d2 - c1 d1 - e p
//   d2 = d2 + t;  d1 = g d1 + d2;  p = g p + d1;   output p
// With g = 1 this is A_i X + b_i x, A_i the one-step matrix of rf_coef.cuh.
//
// Transposed step (third order), costate (lp, l1, l2) of (p, d1, d2), input
// y (zero at land): the exact transpose of the forward step written as the
// reversed sequence of its elementary operations,
//   lp = g lp + y;  l1 = g l1 + lp;  l2 = g l2 + l1;  output beta l2
//   lp -= e l2;  l1 -= c1 l2;  l2 -= c2 l2
// which equals A_i^T acting on the costate after adding y, with output
// beta (lp + l1 + l2).
//
// The steps are written once over a "lane value" type: one FP32 value, or a
// pair of FP32 values from two slices packed in 64 bits and processed with
// the paired FP32 instructions (fma/add/mul .f32x2), so one instruction
// advances two slices.
#pragma once

namespace rfvh {

__device__ __forceinline__ bool right_end(const float4 &c)
{
    return __float_as_uint(c.x) >> 31;
}

// Scalar lane values.
struct V1 {
    using T = float;
    static __device__ __forceinline__ T bc(float a) { return a; }
    static __device__ __forceinline__ T zero() { return 0.f; }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ float get(T a, int) { return a; }
    static __device__ __forceinline__ T make(const float *v) { return v[0]; }
};

// Two slices per 64-bit register.
struct V2 {
    using T = unsigned long long;
    static __device__ __forceinline__ T pack(float a, float b)
    {
        T r;
        asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
        return r;
    }
    static __device__ __forceinline__ T bc(float a) { return pack(a, a); }
    static __device__ __forceinline__ T zero() { return 0ull; }
    static __device__ __forceinline__ T fma(T a, T b, T c)
    {
        T d;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
        return d;
    }
    static __device__ __forceinline__ T add(T a, T b)
    {
        T d;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
        return d;
    }
    static __device__ __forceinline__ T mul(T a, T b)
    {
        T d;
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
        return d;
    }
    static __device__ __forceinline__ float get(T a, int h)
    {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
        return h ? hi : lo;
    }
    static __device__ __forceinline__ T make(const float *v) { return pack(v[0], v[1]); }
};

// Broadcast coefficients of one point for lane-value type L.
template <class L>
struct CoefV {
    typename L::T b, ne, nc1, nc2, g;
    __device__ __forceinline__ CoefV(const float4 &c, float gg)
        : b(L::bc(c.x)), ne(L::bc(c.y)), nc1(L::bc(c.z)), nc2(L::bc(c.w)), g(L::bc(gg))
    {
    }
};

// One step of the sweep kind selected at compile time.  s[0..2] is the
// (co)state; for order 1 only s[0] is used.
template <class L, int ORDER, bool ADJ>
__device__ __forceinline__ typename L::T stepv(typename L::T x, const CoefV<L> &c,
                                               typename L::T *s)
{
    using T = typename L::T;
    if (ORDER == 3) {
        if (!ADJ) {
            T t = L::mul(c.b, x);
            t = L::fma(c.nc2, s[2], t);
            t = L::fma(c.nc1, s[1], t);
            t = L::fma(c.ne, s[0], t);
            s[2] = L::add(s[2], t);
            s[1] = L::fma(c.g, s[1], s[2]);
            s[0] = L::fma(c.g, s[0], s[1]);
            return s[0];
        }
        s[0] = L::fma(c.g, s[0], x);
        s[1] = L::fma(c.g, s[1], s[0]);
        s[2] = L::fma(c.g, s[2], s[1]);
        const T out = L::mul(c.b, s[2]);
        s[0] = L::fma(c.ne, s[2], s[0]);
        s[1] = L::fma(c.nc1, s[2], s[1]);
        s[2] = L::fma(c.nc2, s[2], s[2]);
        return out;
    }
    // first order (Sec. 3.1): t = beta x - e p; p = g p + t
    if (!ADJ) {
        const T t = L::fma(c.ne, s[0], L::mul(c.b, x));
        s[0] = L::fma(c.g, s[0], t);
        return s[0];
    }
    s[0] = L::fma(c.g, s[0], x);
    const T out = L::mul(c.b, s[0]);
    s[0] = L::fma(c.ne, s[0], s[0]);
    return out;
}

// Scalar step on a stored coefficient (sign flag already stripped).
template <int ORDER, bool ADJ>
__device__ __forceinline__ float step(float x, const float4 &c, float *s)
{
    const CoefV<V1> cv(c, c.x != 0.f ? 1.f : 0.f);
    return stepv<V1, ORDER, ADJ>(x, cv, s);
}

// Sum of three products m_k x_k, each m_k given as an unevaluated FP32 pair
// hi + lo, by Dot2 of Ogita, Rump & Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26, 2005): the products' rounding errors (by FMA) and
// the additions' rounding errors (by Knuth's TwoSum) are carried in a second
// accumulator, so the result is as accurate as if it were computed in twice
// the working precision and rounded once.  FP32 only: on this part FP64
// issues at a small fraction of the FP32 rate.
__device__ __forceinline__ float dot2_3(float2 m0, float2 m1, float2 m2, float x0, float x1,
                                        float x2)
{
    float p = __fmul_rn(m0.x, x0);
    float e = __fmaf_rn(m0.x, x0, -p);
    e = __fmaf_rn(m0.y, x0, e);
    const float2 m[2] = {m1, m2};
    const float x[2] = {x1, x2};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float h = __fmul_rn(m[k].x, x[k]);
        const float r = __fmaf_rn(m[k].x, x[k], -h);
        const float s = __fadd_rn(p, h);
        const float z = __fsub_rn(s, p);
        const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(s, z)), __fsub_rn(h, z));
        e = __fadd_rn(e, __fadd_rn(q, r));
        e = __fmaf_rn(m[k].y, x[k], e);
        p = s;
    }
    return __fadd_rn(p, e);
}

// Coastal boundary map: forward Y = M X, adjoint Y = M^T X.  M is stored
// row-major as nine hi/lo FP32 pairs of the FP64 map.
template <int ORDER, bool ADJ>
__device__ __forceinline__ void apply_tail(const float2 *M, const float *X, float *Y)
{
    if (ORDER == 3) {
        const float x0 = X[0], x1 = X[1], x2 = X[2];
        float v[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            v[r] = ADJ ? dot2_3(M[r], M[3 + r], M[6 + r], x0, x1, x2)
                       : dot2_3(M[3 * r], M[3 * r + 1], M[3 * r + 2], x0, x1, x2);
#pragma unroll
        for (int r = 0; r < 3; ++r) Y[r] = v[r];
    } else {
        const float p = __fmul_rn(M[0].x, X[0]);
        Y[0] = __fadd_rn(p, __fmaf_rn(M[0].y, X[0], __fmaf_rn(M[0].x, X[0], -p)));
    }
}

}  // namespace rfvh
