// rf_line.cuh -- long-line path: one thread per (line, slice), sequential
// causal then anticausal sweeps straight from global memory.  Used only for
// lines whose tile (coefficients, boundary maps, data) does not fit the tile
// kernel; same coefficients, boundary maps and step functions as the tile
// kernel.  The anticausal start states of the segment ends go through a
// global scratch array indexed by slice and boundary-map index.  With
// constant-extension coasts (cvec non-null) the causal state entering a
// segment starts from x_a s and the backward start state gains x_e m
// (forward); the adjoint adds s.costate and m.lambda to the outputs at the
// segment's first and last points (see rf_tile.cuh).  With carried coasts
// (carry non-null, 1st-RF, K iterations) a segment's record also keeps the
// state entering it and the boundary states of every iteration: iteration
// k starts the segment from sum_d lambda_d S_{k-d} and its backward sweep
// from M X_k + sum_d mu_d X_{k-d} (rf_coef.cuh, carry_weights_fp64).
#pragma once
#include <cstdint>

#include "rf_steps.cuh"

namespace rfvh {

struct LineArgs {
    const float *in;
    float *out;
    const float4 *coef;       // [ncl][nlines][n]
    const int32_t *tail_base; // [ncl*nlines + 1]
    const float2 *tmap;       // [ntail][9] hi/lo pairs
    const float4 *cvec;       // [ntail][2] (m, s) of constant-extension coasts, or null
    float *tscr;              // [nvar*nz][ntail][nr]
    int nr;                   // floats per record: 3, 4 with cvec, 2 + 2 kc with carry
    const float *carry;       // [ntail][2][kc - 1] (mu, lambda) of this direction, or null
    int kc;                   // K of the carried coasts
    int64_t n, nlines, pt_stride, line_stride, plane, ntail, ncl;
    int64_t nz, nvar;         // levels and variables of the field
    int64_t k0, nk;           // this launch filters levels k0 .. k0+nk-1
    int iters;
};

template <int ORDER, bool ADJ>
__global__ void __launch_bounds__(128) line_kernel(LineArgs a)
{
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= a.nlines * a.nvar * a.nk) return;
    const int64_t item = gid / a.nlines, line = gid - item * a.nlines;
    const int64_t slice = (item / a.nk) * a.nz + a.k0 + item % a.nk;
    const int64_t lev = a.ncl > 1 ? slice % a.nz : 0;
    const float4 *cf = a.coef + (lev * a.nlines + line) * a.n;
    const int64_t base = a.ntail > 0 ? a.tail_base[lev * a.nlines + line] : 0;
    const float *src0 = a.in + slice * a.plane + line * a.line_stride;
    float *out = a.out + slice * a.plane + line * a.line_stride;
    const int nr = a.nr;
    float *scr = a.tscr + slice * a.ntail * nr;
    const int64_t n = a.n, ps = a.pt_stride;
    const bool cst = a.cvec != nullptr && a.ntail > 0;
    const float4 *cv = cst ? a.cvec + 2 * base : nullptr;   // this line's segments
    const bool car = a.carry != nullptr && a.ntail > 0;
    const int km = a.kc - 1;
    // carried-coast record: [0] backward start state, [1] state entering
    // the segment, [2, 2 + kc) the end's states X, [2 + kc, 2 + 2 kc) the
    // start's states S
    for (int it = 0; it < a.iters; ++it) {
        const float *src = it == 0 ? src0 : out;
        float st[3] = {0.f, 0.f, 0.f};
        int64_t rk = base;
        bool prev_sea = false;
        for (int64_t k = 0; k < n; ++k) {
            float4 c = cf[k];
            const bool re = right_end(c);
            c.x = fabsf(c.x);
            const bool sea = c.x != 0.f;
            const float x = sea ? src[k * ps] : 0.f;
            if (!ADJ && cst && sea && !prev_sea) {
                // a segment starts: rk counts the segments before it
                const float4 s = cv[2 * (rk - base) + 1];
                st[0] = x * s.x;
                st[1] = x * s.y;
                st[2] = x * s.z;
            }
            if (car && sea && !prev_sea) st[0] = it == 0 ? 0.f : scr[nr * rk + 1];
            prev_sea = sea;
            out[k * ps] = step<ORDER, ADJ>(x, c, st);
            if (re && a.ntail > 0) {
                float *rec = scr + nr * rk;
                if (cst && ADJ) {
                    const float4 m = cv[2 * (rk - base)];
                    rec[3] = ORDER == 3 ? fmaf(m.x, st[0], fmaf(m.y, st[1], m.z * st[2]))
                                        : m.x * st[0];
                }
                apply_tail<ORDER, ADJ>(a.tmap + 9 * rk, st, rec);
                if (car) {
                    rec[2 + it] = st[0];
                    const float *mu = a.carry + 2 * km * rk;
                    for (int d = 1; d <= it; ++d) rec[0] = fmaf(mu[d - 1], rec[2 + it - d], rec[0]);
                }
                if (cst && !ADJ) {
                    const float4 m = cv[2 * (rk - base)];
                    rec[0] = fmaf(x, m.x, rec[0]);
                    if (ORDER == 3) {
                        rec[1] = fmaf(x, m.y, rec[1]);
                        rec[2] = fmaf(x, m.z, rec[2]);
                    }
                }
                ++rk;
            }
        }
        st[0] = st[1] = st[2] = 0.f;
        float extra = 0.f;
        for (int64_t k = n - 1; k >= 0; --k) {
            float4 c = cf[k];
            extra = 0.f;
            if (right_end(c)) {
                if (a.ntail > 0) {
                    --rk;
                    st[0] = scr[nr * rk];
                    st[1] = ORDER == 3 ? scr[nr * rk + 1] : 0.f;
                    st[2] = ORDER == 3 ? scr[nr * rk + 2] : 0.f;
                    if (cst && ADJ) extra = scr[nr * rk + 3];
                } else {
                    st[0] = st[1] = st[2] = 0.f;
                }
                c.x = fabsf(c.x);
            }
            float y = step<ORDER, ADJ>(out[k * ps], c, st) + extra;
            if (ADJ && cst && c.x != 0.f && (k == 0 || cf[k - 1].x == 0.f)) {
                // the segment's first point: rk is its segment's index
                const float4 s = cv[2 * (rk - base) + 1];
                y = fmaf(s.x, st[0], y);
                if (ORDER == 3) y = fmaf(s.y, st[1], fmaf(s.z, st[2], y));
            }
            if (car && c.x != 0.f && (k == 0 || cf[k - 1].x == 0.f) && it + 1 < a.kc) {
                // the segment's first point: keep S and form the next
                // iteration's entering state
                float *rec = scr + nr * rk;
                rec[2 + a.kc + it] = st[0];
                const float *lam = a.carry + 2 * km * rk + km;
                float h = 0.f;
                for (int d = 1; d <= it + 1; ++d) h = fmaf(lam[d - 1], rec[2 + a.kc + it + 1 - d], h);
                rec[1] = h;
            }
            out[k * ps] = y;
        }
    }
}

}  // namespace rfvh
