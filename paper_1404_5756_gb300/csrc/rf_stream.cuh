// rf_stream.cuh -- streaming column kernel: the y pass of the third-order
// filter on level-independent coefficients, one thread per (column, slice
// pair), whole columns, no chunks and no scan.
//
// A warp takes 32 adjacent columns of one slice pair, so every access is a
// coalesced 128-byte row segment.  The first sweep walks the column down,
// reading the input and the row-major coefficients ([n][ncols] float4,
// L2-resident) D rows ahead through a register ring, writes its state to the
// output and keeps the state after each segment end in a per-thread record in
// shared memory.  The coastal maps turn the records into the start states of
// the second sweep (FP64-built maps applied in compensated FP32).  The second
// sweep walks back up, reading the first sweep's output, and writes the
// result.  The record traffic is branch-free: the first sweep stores its
// state every step (to the next record at a segment end, else to a scratch
// slot) and the second sweep reloads the next record every step and selects
// it at a segment end, so the sweeps' code has no data-dependent branches and
// no segment end waits on a load.  The first sweep's output thus makes one
// round trip through memory between the sweeps, in exchange for no chunk
// re-sweeps, no scans and no barriers.  The forward operator runs the causal sweep
// first; the adjoint runs the transposed steps in the same order (the
// transposed anticausal sweep first, walking down) with the transposed maps.
// Land carries (0, 0, 0, -1) with the reset factor g = 0; the sign of beta
// marks a segment's last sea point.
#pragma once
#include <cstdint>

#include "rf_reg.cuh"

namespace rfvh {

constexpr int kStreamMaxEnds = 13;   // segment ends per column the records hold
constexpr int kStreamWarps = 4;      // warps per CTA (slice pairs per CTA)
constexpr int kStreamThreads = kStreamWarps * 32;

// Dynamic shared memory of a launch whose domains have at most `ends`
// segment ends per column: that many records and one scratch slot, 3 u64
// per slot and thread, thread-fastest (bank-conflict free); at most 43 KB
// per CTA.  Sizing it to the domains' own ends leaves the rest of the SM's
// memory to L1, which keeps the coefficient rows the CTAs share.
inline size_t stream_smem_bytes(int ends)
{
    return (size_t)3 * (ends + 1) * kStreamThreads * sizeof(uint64_t);
}

struct StreamArgs {
    const float *in;
    float *out;
    const float4 *coef;       // [n][ncols] (beta with the end flag in its sign, -e, -c1, -c2)
    const int32_t *tail_base; // [ncols + 1] first coastal map of each column
    const float2 *tmap;       // [ntail][9] hi/lo pairs, or null (no imaginary points)
    int64_t n, ncols;         // column length, columns (= the row length nx)
    int64_t plane;            // floats per slice
    int64_t nz, k0, nk;       // slices of this launch: (s / nk) * nz + k0 + s % nk
    int64_t nslices, npairs;  // slices, ceil(nslices / 2)
    int scratch;              // scratch record slot = most segment ends per column (<= kStreamMaxEnds)
};

__device__ __forceinline__ float4 stream_ldc(const float4 *p)
{
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ float stream_ldf(const float *p)
{
    float v;
    asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// One sweep of the column.  DOWN walks rows 0 .. n-1.  FIRST: the sweep
// reads the input (land zeroed) and records the state after each segment
// end in record nr (counting nr up); else it reads the first sweep's output
// and injects record --nr before each segment end.  Both write their
// outputs.  Record e of this thread, component q: sr[(3 e + q) kStreamThreads].
// Running pointers (one row per step) keep the register count low; the ring
// holds the next D rows' coefficients and inputs.
template <bool ADJ, bool DOWN, bool FIRST, int D>
__device__ __forceinline__ void stream_sweep(const float4 *__restrict__ cp, int64_t ncols,
                                             const float *src0, const float *src1, float *dst0,
                                             float *dst1, bool ok1, int n, u64 *sr, int scratch,
                                             int &nr)
{
    const int64_t step = DOWN ? ncols : -ncols;
    const int64_t start = DOWN ? 0 : (int64_t)(n - 1) * ncols;
    const float4 *pc = cp + start;
    const float *p0 = src0 + start, *p1 = src1 + start;
    float *w0 = dst0 + start, *w1 = dst1 + start;
    u64 st[3] = {0ull, 0ull, 0ull};
    u64 nx[3] = {0ull, 0ull, 0ull};
    if (!FIRST) {
        const int e = nr > 0 ? nr - 1 : 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) nx[q] = sr[(3 * e + q) * kStreamThreads];
    }
    const u64 one = V2::bc(1.f);
    float4 rc[D];
    float r0[D], r1[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        if (d < n) {
            rc[d] = stream_ldc(pc);
            r0[d] = stream_ldf(p0);
            r1[d] = ok1 ? stream_ldf(p1) : 0.f;
            pc += step;
            p0 += step;
            p1 += step;
        }
    }
    for (int i0 = 0; i0 < n; i0 += D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int i = i0 + d;
            if (i >= n) break;
            float4 c = rc[d];
            const float u = r0[d], w = r1[d];
            if (i + D < n) {
                rc[d] = stream_ldc(pc);
                r0[d] = stream_ldf(p0);
                r1[d] = ok1 ? stream_ldf(p1) : 0.f;
                pc += step;
                p0 += step;
                p1 += step;
            }
            const bool end = __float_as_uint(c.x) >> 31;
            c.x = fabsf(c.x);
            const bool sea = c.x != 0.f;
            if (!FIRST) {
#pragma unroll
                for (int q = 0; q < 3; ++q) st[q] = end ? nx[q] : st[q];
                nr -= end;
                const int e = nr > 0 ? nr - 1 : 0;
#pragma unroll
                for (int q = 0; q < 3; ++q) nx[q] = sr[(3 * e + q) * kStreamThreads];
            }
            const u64 g = sea ? one : 0ull;
            const u64 x = FIRST ? V2::pack(sea ? u : 0.f, sea ? w : 0.f) : V2::pack(u, w);
            const u64 b = V2::bc(c.x), ne = V2::bc(c.y), n1 = V2::bc(c.z), n2 = V2::bc(c.w);
            const u64 y = ADJ ? rstep_a<3>(x, b, ne, n1, n2, g, st) : rstep_f<3>(x, b, ne, n1, n2, g, st);
            *w0 = V2::get(y, 0);
            if (ok1) *w1 = V2::get(y, 1);
            w0 += step;
            w1 += step;
            if (FIRST) {
                const bool keep = end && nr < scratch;
                const int e = keep ? nr : scratch;
#pragma unroll
                for (int q = 0; q < 3; ++q) sr[(3 * e + q) * kStreamThreads] = st[q];
                nr += keep;
            }
        }
    }
}

// The work of CTA (bx, by) of one domain's grid (stream_grid).
template <bool ADJ, int D>
__device__ __forceinline__ void stream_body(const StreamArgs &a, unsigned bx, unsigned by)
{
    const int64_t col = (int64_t)bx * 32 + (threadIdx.x & 31);
    const int64_t pr = (int64_t)by * kStreamWarps + (threadIdx.x >> 5);
    if (col >= a.ncols || pr >= a.npairs) return;   // no barriers in this kernel
    const int64_t s0 = 2 * pr, s1 = 2 * pr + 1;
    const bool ok1 = s1 < a.nslices;
    const int64_t o0 = ((s0 / a.nk) * a.nz + a.k0 + s0 % a.nk) * a.plane;
    const int64_t o1 = ok1 ? ((s1 / a.nk) * a.nz + a.k0 + s1 % a.nk) * a.plane : o0;
    const float4 *cp = a.coef + col;
    extern __shared__ u64 stream_srec[];   // stream_smem_bytes(scratch of the launch's domains)
    u64 *sr = stream_srec + threadIdx.x;
    int nr = 0;
    // first sweep: down, recording the states at the segment ends
    stream_sweep<ADJ, true, true, D>(cp, a.ncols, a.in + o0 + col, a.in + o1 + col, a.out + o0 + col,
                                     a.out + o1 + col, ok1, (int)a.n, sr, a.scratch, nr);
    // the coastal maps of the column's ends, in order (zero start states
    // without imaginary points)
    const float2 *ml = a.tmap ? a.tmap + 9 * (int64_t)a.tail_base[col] : nullptr;
    for (int q = 0; q < nr; ++q) {
        u64 r[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] = sr[(3 * q + k) * kStreamThreads];
        if (!ml) {
            r[0] = r[1] = r[2] = 0ull;
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float X[3], Y[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) X[k] = V2::get(r[k], h);
                apply_tail<3, ADJ>(ml + 9 * q, X, Y);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float lo = V2::get(r[k], 0), hi = V2::get(r[k], 1);
                    if (h == 0) lo = Y[k];
                    else hi = Y[k];
                    r[k] = V2::pack(lo, hi);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) sr[(3 * q + k) * kStreamThreads] = r[k];
    }
    // second sweep: up, from the first sweep's output in place
    stream_sweep<ADJ, false, false, D>(cp, a.ncols, a.out + o0 + col, a.out + o1 + col, a.out + o0 + col,
                                       a.out + o1 + col, ok1, (int)a.n, sr, a.scratch, nr);
}

template <bool ADJ, int D>
__global__ void __launch_bounds__(kStreamWarps * 32) stream_kernel(const StreamArgs a)
{
    stream_body<ADJ, D>(a, blockIdx.x, blockIdx.y);
}

// One launch over several domains (a ragged batch): the 1-D grid is the
// concatenation of the domains' grids; cta0[d] is the first CTA of domain d,
// gx[d] the x extent of its grid.
constexpr int kStreamMulti = 64;
struct StreamMulti {
    int nd;
    int gx[kStreamMulti];
    int64_t cta0[kStreamMulti + 1];
    StreamArgs dom[kStreamMulti];
};

template <bool ADJ, int D>
__global__ void __launch_bounds__(kStreamWarps * 32) stream_multi_kernel(const __grid_constant__ StreamMulti m)
{
    const int64_t b = blockIdx.x;
    int lo = 0, hi = m.nd - 1;   // the domain d with cta0[d] <= b < cta0[d + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m.cta0[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int64_t r = b - m.cta0[lo];
    stream_body<ADJ, D>(m.dom[lo], (unsigned)(r % m.gx[lo]), (unsigned)(r / m.gx[lo]));
}

}  // namespace rfvh
