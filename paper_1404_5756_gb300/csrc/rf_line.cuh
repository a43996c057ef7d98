// rf_line.cuh -- long-line path: one thread per (line, slice), sequential
// causal then anticausal sweeps straight from global memory.  Used only for
// lines whose tile (coefficients, boundary maps, data) does not fit the tile
// kernel; same coefficients, boundary maps and step functions as the tile
// kernel.  The anticausal start states of the segment ends go through a
// global scratch array indexed by slice and boundary-map index.
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
    float *tscr;              // [nvar*nz][ntail][3]
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
    float *scr = a.tscr + slice * a.ntail * 3;
    const int64_t n = a.n, ps = a.pt_stride;
    for (int it = 0; it < a.iters; ++it) {
        const float *src = it == 0 ? src0 : out;
        float st[3] = {0.f, 0.f, 0.f};
        int64_t rk = base;
        for (int64_t k = 0; k < n; ++k) {
            float4 c = cf[k];
            const bool re = right_end(c);
            c.x = fabsf(c.x);
            const float x = c.x != 0.f ? src[k * ps] : 0.f;
            out[k * ps] = step<ORDER, ADJ>(x, c, st);
            if (re && a.ntail > 0) {
                apply_tail<ORDER, ADJ>(a.tmap + 9 * rk, st, scr + 3 * rk);
                ++rk;
            }
        }
        st[0] = st[1] = st[2] = 0.f;
        for (int64_t k = n - 1; k >= 0; --k) {
            float4 c = cf[k];
            if (right_end(c)) {
                if (a.ntail > 0) {
                    --rk;
                    st[0] = scr[3 * rk];
                    st[1] = ORDER == 3 ? scr[3 * rk + 1] : 0.f;
                    st[2] = ORDER == 3 ? scr[3 * rk + 2] : 0.f;
                } else {
                    st[0] = st[1] = st[2] = 0.f;
                }
                c.x = fabsf(c.x);
            }
            out[k * ps] = step<ORDER, ADJ>(out[k * ps], c, st);
        }
    }
}

}  // namespace rfvh
