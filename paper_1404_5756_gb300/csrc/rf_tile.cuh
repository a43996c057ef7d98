// rf_tile.cuh -- the main filter kernel: R whole lines per CTA, P lanes per
// line (P = 32: one line per warp; P = 16: two lines per warp, for short
// lines), the P lanes of a line owning consecutive chunks of C points (C odd,
// P*C >= n, C <= 128).  Each thread filters B slices of its chunk at once (B
// independent recursions: instruction-level parallelism, and one coefficient
// read serves B slices).  The line data of the B slices and the coastal
// boundary maps of the CTA's lines sit in shared memory; the per-point
// coefficients are read from global memory in a lane-interleaved layout
// (step j of all P lanes of a line is one contiguous row, so every read is
// coalesced; the rows are re-read by each sweep and slice group, mostly from
// L2, three steps ahead of their use).  The chunk carries are
// resolved with a Kogge-Stone scan of affine maps over the lanes (warp
// shuffles).  One kernel serves both directions:
//   x pass: a line is a row, points contiguous in global memory;
//   y pass: a line is a column, points nx apart; R adjacent columns are
//           loaded together so each row segment is R*4 contiguous bytes.
//
// Per line and slice (a slice is one level of one variable), for each of the
// K iterations (K = 1 for the third-order filter):
//   A  causal sweep of every chunk from zero state -> chunk end state
//   scan of (Phi_chunk, end state) over the lanes -> true state at each chunk
//   B  causal sweep again from the true state -> causal output (in place),
//      recording the causal state at the last sea point of every segment;
//      the warp then turns each into the anticausal start state with the
//      segment's coastal boundary map (built in FP64, applied in compensated
//      FP32)
//   C  anticausal sweep from zero state (boundary-map starts included)
//   scan in the reverse lane order
//   D  anticausal sweep from the true state -> final output (in place)
// The forward operator uses the forward steps, the adjoint the transposed
// steps; the chunk transfer matrices Phi come precomputed from the plan.
//
// Constant-extension coasts (CST kernels, an option): the imaginary points
// carry the segment's edge values.  Forward: at a segment's first sea point
// the causal state starts from x_a s (A and B), and the backward start state
// gains x_e m (the last input x_e is recorded with the causal state in B).
// Adjoint: the transposed terms, s.lambda and m.lambda, are added to the
// outputs at the segment's first and last points in D.  s and m are
// per-segment FP32 vectors built in FP64 by the plan.
#pragma once
#include <cstdint>

#include "rf_steps.cuh"

namespace rfvh {

// Segment ends of one chunk: bit j marks point j.  Bits64 serves chunks of
// up to 64 points (the common case, one 64-bit word), SegBits chunks of up
// to 128 (lo: points 0..63, hi: 64..127); both give the sweeps the same
// interface.
struct Bits64 {
    unsigned long long v;
    __device__ __forceinline__ int first() const { return v ? __ffsll((long long)v) - 1 : 64; }
    __device__ __forceinline__ int last() const { return v ? 63 - __clzll((long long)v) : -1; }
    __device__ __forceinline__ void drop_first() { v &= v - 1; }
    __device__ __forceinline__ void drop(int j) { v &= ~(1ull << j); }
    __device__ __forceinline__ int count() const { return __popcll((long long)v); }
};

struct SegBits {
    unsigned long long lo, hi;
    __device__ __forceinline__ int first() const   // lowest marked point, 128 if none
    {
        return lo ? __ffsll((long long)lo) - 1 : hi ? 63 + __ffsll((long long)hi) : 128;
    }
    __device__ __forceinline__ int last() const    // highest marked point, -1 if none
    {
        return hi ? 127 - __clzll((long long)hi) : lo ? 63 - __clzll((long long)lo) : -1;
    }
    __device__ __forceinline__ void drop_first()
    {
        if (lo) lo &= lo - 1;
        else hi &= hi - 1;
    }
    __device__ __forceinline__ void drop(int j)
    {
        if (j < 64) lo &= ~(1ull << j);
        else hi &= ~(1ull << (j - 64));
    }
    __device__ __forceinline__ int count() const
    {
        return __popcll((long long)lo) + __popcll((long long)hi);
    }
};

// Per (line, lane) record of the segment ends and starts in the lane's chunk.
struct LaneInfo {
    SegBits re;    // segment ends in the chunk
    int rank0;     // segment ends on the line before this chunk
    int nre;       // segment ends in this chunk
    SegBits rs;    // segment starts (first sea point of a run) in the chunk
    int rs0;       // segment starts on the line before this chunk
    int pad;
};

struct TileArgs {
    const float *in;          // field [nslices][...] of this domain
    float *out;
    const float4 *coef;       // [ncl][nlines][C][P] interleaved (beta, -e, -c1, -c2)
    const LaneInfo *lanes;    // [ncl][nlines][P]
    const float *xfer;        // [ncl][nlines][P][XF] chunk transfers
    const int32_t *tail_base; // [ncl*nlines + 1] index of each line's first boundary map
    const float2 *tmap;       // [ntail][9] hi/lo pairs, consecutive along each line
    const float4 *cvec;       // [ntail][2] (m, s) of constant-extension coasts, or null
    int64_t n, nlines;        // line length, lines per slice
    int64_t pt_stride;        // distance between consecutive points of a line
    int64_t line_stride;      // distance between consecutive lines
    int64_t plane;            // floats per slice
    int64_t nz;               // levels of the field
    int64_t nvar;             // variables of the field
    int64_t k0, nk;           // this launch filters levels k0 .. k0+nk-1
    int64_t ncl;              // coefficient levels (1 or nz)
    int C;                    // chunk length (odd, <= 128)
    int iters;
    int smem_stride;          // floats per line row in shared memory
    int max_re;               // boundary-map slots per line (0: no maps)
    int vec4;                 // 16-byte aligned rows (x pass) or grid rows (y pass)
    int nbuf;                 // data buffers: 1 or 2 (copies overlap filtering)
};

constexpr int kMaxChunk = 128;
// float4 guard entries before and after the interleaved coefficient array,
// so the sweeps may prefetch up to three steps past either end of a chunk
// (3 x 32 lanes)
constexpr int kCoefGuard = 128;

// Transfer record per chunk: order 3 -> four 3x3 row-major matrices
// (forward causal, forward anticausal, adjoint causal, adjoint anticausal);
// order 1 -> four scalars.
template <int ORDER>
struct XF {
    static constexpr int size = ORDER == 3 ? 36 : 4;
    static constexpr int mat = ORDER == 3 ? 9 : 1;
};

__device__ __forceinline__ void cp_async4(void *s, const void *g)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(g));
}

__device__ __forceinline__ void cp_async8(void *s, const void *g)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(g));
}

__device__ __forceinline__ void cp_async16(void *s, const void *g)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(g));
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int ORDER>
__device__ __forceinline__ void mat_vec(const float *P, const float *v, float *o)
{
    if (ORDER == 3) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
            o[r] = fmaf(P[3 * r], v[0], fmaf(P[3 * r + 1], v[1], P[3 * r + 2] * v[2]));
    } else {
        o[0] = P[0] * v[0];
    }
}

template <int ORDER>
__device__ __forceinline__ void mat_mat(const float *P, const float *Q, float *o)
{
    if (ORDER == 3) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                o[3 * r + c] = fmaf(P[3 * r], Q[c], fmaf(P[3 * r + 1], Q[3 + c], P[3 * r + 2] * Q[6 + c]));
    } else {
        o[0] = P[0] * Q[0];
    }
}

// Exclusive scan of affine maps over the P lanes of a line (segments of P
// lanes of the warp), for B slices sharing the maps' linear parts.  Lane l of
// the line holds x -> Pm x + v[b].  Forward (REV = false): lane l receives the
// state entering its chunk from lanes 0..l-1; REV: from lanes P-1..l+1.
template <int ORDER, bool REV, int B, int P>
__device__ __forceinline__ void warp_scan(float *Pm, float (*v)[3], int lane)
{
    constexpr int M = XF<ORDER>::mat;
    constexpr int S = ORDER == 3 ? 3 : 1;
#pragma unroll
    for (int d = 1; d < P; d <<= 1) {
        float Pn[M], vn[B][S];
#pragma unroll
        for (int k = 0; k < M; ++k)
            Pn[k] = REV ? __shfl_down_sync(0xffffffffu, Pm[k], d, P)
                        : __shfl_up_sync(0xffffffffu, Pm[k], d, P);
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int k = 0; k < S; ++k)
                vn[b][k] = REV ? __shfl_down_sync(0xffffffffu, v[b][k], d, P)
                               : __shfl_up_sync(0xffffffffu, v[b][k], d, P);
        const bool take = REV ? (lane + d < P) : (lane >= d);
        if (take) {
#pragma unroll
            for (int b = 0; b < B; ++b) {
                float nv[S];
                mat_vec<ORDER>(Pm, vn[b], nv);
#pragma unroll
                for (int k = 0; k < S; ++k) v[b][k] += nv[k];
            }
            if (2 * d < P) {   // the last level's composed map is never used
                float nP[M];
                mat_mat<ORDER>(Pm, Pn, nP);
#pragma unroll
                for (int k = 0; k < M; ++k) Pm[k] = nP[k];
            }
        }
    }
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const float t = REV ? __shfl_down_sync(0xffffffffu, v[b][k], 1, P)
                                : __shfl_up_sync(0xffffffffu, v[b][k], 1, P);
            v[b][k] = (REV ? lane == P - 1 : lane == 0) ? 0.f : t;
        }
}

// Shared-memory bytes of the tile kernel.  Layout: 16-byte guard | maps
// [R][max_re][9] float2 (padded to 16 bytes) | nbuf data buffers (1 or 2),
// each [B/W][R][ss] units of W slices | starts [B][R][max_re][nr] float
// (nr = 3, or 4 with constant-extension coasts) | 16-byte guard.  The guards
// keep the sweeps' one-step-ahead data prefetch (one element past either end
// of a chunk) inside the allocation.
__host__ __device__ inline int64_t tile_smem_bytes(int64_t R, int64_t B, int64_t ss,
                                                   int64_t max_re, int64_t nbuf, int64_t nr = 3)
{
    const int64_t maps = (R * max_re * 9 + 1) / 2 * 2;
    return 16 + maps * 8 + nbuf * B * R * ss * 4 + B * R * max_re * nr * 4 + 16;
}

// B slices per thread travel as U = B/W lane values of W slices each: pairs
// (packed FP32x2 arithmetic) when B is even.
template <int B>
struct Pack {
    static constexpr int W = B % 2 == 0 ? 2 : 1;
    static constexpr int U = B / W;
};
template <int W>
struct LaneT;
template <>
struct LaneT<1> {
    using L = V1;
};
template <>
struct LaneT<2> {
    using L = V2;
};

// One sweep over a lane's chunk for B slices.  cp points at the chunk's
// first coefficient (consecutive steps P float4 apart), dp[u] at lane value
// u's first data element, len points.  CAUSAL walks up, else down.  IN_SEA
// zeroes the input at land and writes the zero back (first read of the
// data); WRITE stores the outputs in place.  rebits marks segment ends (bit
// j <-> point j).  In a causal sweep with TAILS the state after a segment end
// is recorded for the boundary map (at ys[b] + NR*rank, rank counting up from
// rk); in an anticausal sweep the state is reset to the stored start state
// before the segment end is stepped (rank counting down from rk), or to zero
// without maps.  Coefficients are fetched three steps ahead and data one step
// ahead, so memory latency overlaps the arithmetic.
//
// CST (constant-extension coasts; the records are NR = 4 floats): rsbits
// marks segment starts, their vectors (m, s) at cv[2 rank], rank counting up
// from sk (causal) or down (anticausal).  Forward causal: the state entering
// a start is x s, and B records the input at a segment end in the fourth
// float.  Adjoint anticausal with WRITE: the output at a segment end gains
// the fourth float of its record (m.lambda, from the tails), the output at a
// start gains s.costate.
template <int ORDER, bool ADJ, int B, int P, bool CAUSAL, bool IN_SEA, bool WRITE, bool TAILS,
          bool CST, class MASK>
__device__ __forceinline__ void sweep(const float4 *__restrict__ cp,
                                      typename LaneT<Pack<B>::W>::L::T *const *dp, int len,
                                      MASK rebits, MASK rsbits, const float4 *__restrict__ cv,
                                      int sk, float *const *ys, int rk,
                                      typename LaneT<Pack<B>::W>::L::T (*st)[3])
{
    constexpr int W = Pack<B>::W, U = Pack<B>::U, NS = ORDER == 3 ? 3 : 1;
    constexpr int NR = CST ? 4 : 3;
    // start events: forward causal sweeps and the adjoint's writing anticausal one
    constexpr bool STARTS = CST && (CAUSAL ? !ADJ : (ADJ && WRITE));
    constexpr bool EXTRA = CST && !CAUSAL && ADJ && WRITE && TAILS;
    // a causal sweep that records nothing and starts nothing has no events
    // (the zero-start sweep A): no per-step test
    constexpr bool ENDS = !CAUSAL || TAILS;
    using L = typename LaneT<W>::L;
    using T = typename L::T;
    if (len <= 0) return;   // empty chunk: touch no memory
    const int dir = CAUSAL ? 1 : -1;
    int j = CAUSAL ? 0 : len - 1;
    int re_next, rs_next = -2;
    if (CAUSAL) re_next = rebits.first();
    else re_next = rebits.last();
    if (STARTS) rs_next = CAUSAL ? rsbits.first() : rsbits.last();
    float4 c = __ldg(cp + P * j);
    float4 c1 = __ldg(cp + P * (j + dir));
    float4 c2 = __ldg(cp + P * (j + 2 * dir));
    T x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = dp[u][j];
#pragma unroll 2
    for (int t = 0; t < len; ++t, j += dir) {
        const float4 c3 = __ldg(cp + P * (j + 3 * dir));
        T xn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xn[u] = dp[u][j + dir];
        const bool sea = c.x != 0.f;
        const CoefV<L> cv4(c, sea ? 1.f : 0.f);
        const bool at_end = ENDS && j == re_next;
        const bool at_start = STARTS && j == rs_next;
        T ex[U];
        if (!CAUSAL && at_end) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    float v[W];
#pragma unroll
                    for (int h = 0; h < W; ++h) v[h] = TAILS ? ys[u * W + h][NR * rk + q] : 0.f;
                    st[u][q] = L::make(v);
                }
                if (EXTRA) {
                    float v[W];
#pragma unroll
                    for (int h = 0; h < W; ++h) v[h] = ys[u * W + h][NR * rk + 3];
                    ex[u] = L::make(v);
                }
            }
            if (TAILS) --rk;
        }
        float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (at_start) sv = __ldg(cv + 2 * sk + 1);
        if (CAUSAL && at_start) {
            // the imaginary points before the segment carry its first value
#pragma unroll
            for (int u = 0; u < U; ++u) {
                st[u][0] = L::mul(x[u], L::bc(sv.x));
                if (NS == 3) {
                    st[u][1] = L::mul(x[u], L::bc(sv.y));
                    st[u][2] = L::mul(x[u], L::bc(sv.z));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            T in = x[u];
            if (IN_SEA && !sea) {
                in = L::zero();
                dp[u][j] = in;
            }
            T y = stepv<L, ORDER, ADJ>(in, cv4, st[u]);
            if (EXTRA && at_end) y = L::add(y, ex[u]);
            if (!CAUSAL && at_start) {
                y = L::fma(st[u][0], L::bc(sv.x), y);
                if (NS == 3) {
                    y = L::fma(st[u][1], L::bc(sv.y), y);
                    y = L::fma(st[u][2], L::bc(sv.z), y);
                }
            }
            if (WRITE) dp[u][j] = y;
        }
        if (CAUSAL && TAILS && at_end) {
            // record the final causal state (and, forward CST, the last
            // input); the boundary maps are applied afterwards by the whole
            // warp (apply_line_tails)
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int h = 0; h < W; ++h) {
#pragma unroll
                    for (int q = 0; q < NS; ++q) ys[u * W + h][NR * rk + q] = L::get(st[u][q], h);
                    if (CST && !ADJ) ys[u * W + h][NR * rk + 3] = L::get(x[u], h);
                }
            ++rk;
        }
        if (at_end) {
            if (CAUSAL) {
                rebits.drop_first();
                re_next = rebits.first();
            } else {
                rebits.drop(j);
                re_next = rebits.last();
            }
        }
        if (at_start) {
            if (CAUSAL) {
                rsbits.drop_first();
                rs_next = rsbits.first();
                ++sk;
            } else {
                rsbits.drop(j);
                rs_next = rsbits.last();
                --sk;
            }
        }
        c = c1;
        c1 = c2;
        c2 = c3;
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = xn[u];
    }
}

// Coastal boundary maps of one line, applied by the whole warp after the
// causal sweep: for every segment end q of the line (its P lanes take
// q = lane, lane + P, ...) and every slice b, replace the recorded causal state X at
// ys[b] + NR q by the anticausal start state M_q X (adjoint: M_q^T X).
// Spreading the segment ends over the lanes keeps the compensated map
// arithmetic out of the divergent per-point loop.  CST: forward adds x_e m_q
// (x_e recorded in the fourth float), adjoint stores m_q.X in the fourth
// float for the output at the segment end.
template <int ORDER, bool ADJ, int B, int P, bool CST>
__device__ __forceinline__ void apply_line_tails(const float2 *ml, float *const *ys, int nre_line,
                                                 int lane, const float4 *__restrict__ cv)
{
    constexpr int NS = ORDER == 3 ? 3 : 1;
    constexpr int NR = CST ? 4 : 3;
    __syncwarp();
    for (int q = lane; q < nre_line; q += P) {
        float4 mv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (CST) mv = __ldg(cv + 2 * q);
#pragma unroll
        for (int b = 0; b < B; ++b) {
            float X[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < NS; ++k) X[k] = ys[b][NR * q + k];
            float *Y = ys[b] + NR * q;
            if (CST && ADJ) {
                float d = mv.x * X[0];
                if (NS == 3) d = fmaf(mv.y, X[1], fmaf(mv.z, X[2], d));
                Y[3] = d;
            }
            apply_tail<ORDER, ADJ>(ml + 9 * q, X, Y);
            if (CST && !ADJ) {
                const float xe = Y[3];
                Y[0] = fmaf(xe, mv.x, Y[0]);
                if (NS == 3) {
                    Y[1] = fmaf(xe, mv.y, Y[1]);
                    Y[2] = fmaf(xe, mv.z, Y[2]);
                }
            }
        }
    }
    __syncwarp();
}

// The work of one CTA: line block bx (lines bx*R ..) and CTA row by of gy
// rows along the slices (see the slice mapping below).  R*P threads: line rl
// of the CTA is handled by lanes rl*P .. rl*P + P-1.
template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
__device__ __forceinline__ void tile_body(const TileArgs &a, int64_t bx, int64_t by, int64_t gy,
                                          unsigned char *smem_raw)
{
    constexpr int XS = XF<ORDER>::size, M = XF<ORDER>::mat;
    constexpr int NR = CST ? 4 : 3;   // floats per segment-end record
    constexpr int W = Pack<B>::W, U = Pack<B>::U;
    constexpr int LPW = 32 / P;   // lines per warp
    static_assert(P == 32 || P == 16, "lanes per line");
    static_assert(R % LPW == 0, "whole warps per CTA");
    using L = typename LaneT<W>::L;
    using T = typename L::T;
    const int warp = threadIdx.x >> 5;
    const int rl = threadIdx.x / P, lane = threadIdx.x % P;   // line of the CTA, lane on it
    const int n = (int)a.n, C = a.C, ss = a.smem_stride, mre = a.max_re;
    float2 *ms = reinterpret_cast<float2 *>(smem_raw + 16);
    float *ds = reinterpret_cast<float *>(ms + ((R * mre * 9 + 1) & ~1));
    float *ys = ds + a.nbuf * B * R * ss;   // after the data buffers
    const int64_t line0 = bx * R;
    const int64_t myline = line0 + rl;
    // a warp works if its first line exists; its other lines past the end run
    // on the last line's data (every lane must join the shuffles) and are
    // never stored
    const bool active = line0 + (int64_t)warp * LPW < a.nlines;
    const int64_t lc = min(myline, a.nlines - 1);
    const int lines_here = (int)min((int64_t)R, a.nlines - line0);

    // A launch filters levels k0 .. k0+nk-1 of all nvar variables.  Slices are
    // handled in groups of B sharing one coefficient level.  One level for
    // every slice: item i of the launch is slice (i / nk)*nz + k0 + i % nk,
    // group g holds items g*B + b, and CTA row y takes groups y, y + rows, ...
    // Per-level coefficients: CTA row y is level k0 + y and its groups hold
    // the variables g*B + b of that level.
    const bool one_level = a.ncl == 1;
    const int64_t lev = one_level ? 0 : a.k0 + by;
    const int64_t nvar = a.nvar, nitems = a.nvar * a.nk;
    const int64_t ngroups = one_level ? (nitems + B - 1) / B : (nvar + B - 1) / B;
    const int64_t lvl_lines = lev * a.nlines;

    // boundary maps of the R lines
    if (mre > 0) {
        for (int r = 0; r < lines_here; ++r) {
            const int64_t base = a.tail_base[lvl_lines + line0 + r];
            const int cnt = (int)(a.tail_base[lvl_lines + line0 + r + 1] - base);
            const float2 *g = a.tmap + 9 * base;
            float2 *s = ms + r * mre * 9;
            for (int q = threadIdx.x; q < cnt * 9; q += blockDim.x) cp_async8(s + q, g + q);
        }
    }
    // my chunk [ka, kb); lanes past the line's end get an empty chunk at n
    const int ka = min(lane * C, n), kb = min(ka + C, n), len = kb - ka;
    const float4 *cg = a.coef + ((lvl_lines + lc) * C) * P + lane;
    const float2 *ml = ms + rl * mre * 9;
    SegBits rebits{0ull, 0ull}, rsbits{0ull, 0ull};
    int rank0 = 0, nre = 0, line_re = 0, rs0 = 0;
    const float4 *cvl = nullptr;   // the line's constant-coast vectors
    float Pc[M], Pa[M];
    if (active) {
        const LaneInfo li = a.lanes[(lvl_lines + lc) * P + lane];
        rebits = li.re;
        rank0 = li.rank0;
        nre = li.nre;
        if (CST) {
            rsbits = li.rs;
            rs0 = li.rs0;
        }
        if (mre > 0) {
            line_re = (int)(a.tail_base[lvl_lines + lc + 1] - a.tail_base[lvl_lines + lc]);
            if (CST) cvl = a.cvec + 2 * (int64_t)a.tail_base[lvl_lines + lc];
        }
        const float *x = a.xfer + ((lvl_lines + lc) * P + lane) * XS;
        const int oc = ADJ ? 2 : 0, oa = ADJ ? 3 : 1;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            Pc[k] = x[oc * M + k];
            Pa[k] = x[oa * M + k];
        }
    }
    // data layout: lane value u of line r at T-index (u*R + r)*ss + k, i.e.
    // slice b of line r, point k at float index W*((b/W*R + r)*ss + k) + b%W
    T *dt = reinterpret_cast<T *>(ds);
    T *dl[U];
    float *yl[B];
#pragma unroll
    for (int b = 0; b < B; ++b) yl[b] = ys + (b * R + rl) * mre * NR;
    // load/store mapping: the x pass copies rows, the y pass R-column
    // strips, thread t owning column r = t % R and rows t / R + P m
    const int yr = threadIdx.x % R, yk0 = threadIdx.x / R;
    const int64_t row_step = (int64_t)P * a.pt_stride;
    const bool maps = mre > 0;
    const bool vec = W == 1 && a.vec4 && a.pt_stride == 1;

    // Slice groups of this CTA, double buffered: the copies of the next
    // group are in flight while the current one is filtered.
    const int64_t g_first = one_level ? by : 0;
    const int64_t g_step = one_level ? gy : 1;
    auto slice_of = [&](int64_t gi, int b) -> int64_t {
        const int64_t i = gi * B + b;
        return one_level ? (i / a.nk) * a.nz + a.k0 + i % a.nk : i * a.nz + lev;
    };
    auto group_size = [&](int64_t gi) {
        return (int)min((int64_t)B, one_level ? nitems - gi * B : nvar - gi * B);
    };
    // rows in slice pairs with one buffer: 16-byte loads from both slices of
    // a pair, interleaved in registers into two 16-byte shared stores (the
    // copy engine cannot interleave); otherwise element-wise cp.async
    const bool pv = W == 2 && a.vec4 && a.nbuf == 1 && a.pt_stride == 1;
    // columns in slice pairs: each thread stores 4 adjacent columns of one
    // row of both slices of a pair as two 16-byte stores (4 paired 8-byte
    // shared loads), instead of 8 scalar stores
    const bool svy = W == 2 && a.vec4 && a.pt_stride != 1 && R % 4 == 0;
    constexpr int QY = R >= 4 ? R / 4 : 1;   // column quads per row
    const int cq = threadIdx.x % QY, yk1 = threadIdx.x / QY, ykstep = blockDim.x / QY;
    auto issue_loads = [&](int64_t gi, int buf) {
        const int nb = group_size(gi);
        if (pv) {
            for (int u = 0; u < (nb + 1) / 2; ++u) {
                const float *s0 = a.in + slice_of(gi, 2 * u) * a.plane;
                const float *s1 = 2 * u + 1 < nb ? a.in + slice_of(gi, 2 * u + 1) * a.plane : nullptr;
                float *db = ds + (int64_t)buf * B * R * ss + (int64_t)u * 2 * R * ss;
                for (int r = 0; r < lines_here; ++r) {
                    const float4 *g0 = reinterpret_cast<const float4 *>(s0 + (line0 + r) * a.line_stride);
                    const float4 *g1 = s1 ? reinterpret_cast<const float4 *>(s1 + (line0 + r) * a.line_stride)
                                          : nullptr;
                    float4 *sr = reinterpret_cast<float4 *>(db + 2 * r * ss);
#pragma unroll 8
                    for (int q = threadIdx.x; q < n / 4; q += blockDim.x) {
                        const float4 x0 = __ldg(g0 + q);
                        const float4 x1 = g1 ? __ldg(g1 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                        sr[2 * q] = make_float4(x0.x, x1.x, x0.y, x1.y);
                        sr[2 * q + 1] = make_float4(x0.z, x1.z, x0.w, x1.w);
                    }
                }
            }
            // the boundary-map copies issued earlier join a group, so the
            // wait before filtering covers them
            asm volatile("cp.async.commit_group;\n" ::);
            return;
        }
        for (int b = 0; b < nb; ++b) {
            const float *src = a.in + slice_of(gi, b) * a.plane;
            float *db = ds + (int64_t)buf * B * R * ss + (b / W) * W * R * ss + b % W;
            if (a.pt_stride == 1) {
                for (int r = 0; r < lines_here; ++r) {
                    const float *g = src + (line0 + r) * a.line_stride;
                    float *s = db + W * r * ss;
                    if (vec) {
                        for (int q = threadIdx.x; q < n / 4; q += blockDim.x)
                            cp_async16(s + 4 * q, g + 4 * q);
                    } else {
                        for (int k = threadIdx.x; k < n; k += blockDim.x) cp_async4(s + W * k, g + k);
                    }
                }
            } else if (yr < lines_here) {
                const float *g = src + (line0 + yr) + (int64_t)yk0 * a.pt_stride;
                float *s = db + W * yr * ss;
                for (int k = yk0; k < n; k += P, g += row_step) cp_async4(s + W * k, g);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    // one buffer: copy, filter, store in turn; two: the next group's copies
    // fly while the current group is filtered
    const bool dbl = a.nbuf == 2;
    if (dbl && g_first < ngroups) issue_loads(g_first, 0);
    int buf = 0;
    for (int64_t gi = g_first; gi < ngroups; gi += g_step, buf ^= (dbl ? 1 : 0)) {
        const int nb = group_size(gi);
        if (!dbl) issue_loads(gi, 0);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();   // group gi has landed; the other buffer is free
        if (dbl && gi + g_step < ngroups) issue_loads(gi + g_step, buf ^ 1);
#pragma unroll
        for (int u = 0; u < U; ++u) dl[u] = dt + ((int64_t)buf * U * R + u * R + rl) * ss + ka;
        // the filter work of the group, for the chunk's segment mask type
        auto filter = [&](auto rebits, auto rsbits) {
            using MASK = decltype(rebits);
            // constant-extension coasts need boundary maps (imaginary points)
            const bool cst = CST && maps;
            const int nrs = CST ? rsbits.count() : 0;
            for (int it = 0; it < a.iters; ++it) {
                T st[U][3];
                float v[B][3], Pm[M];
                // ---- A: causal, zero start -> chunk end state (land input zeroed)
#pragma unroll
                for (int u = 0; u < U; ++u) st[u][0] = st[u][1] = st[u][2] = L::zero();
                if (cst && !ADJ)
                    sweep<ORDER, ADJ, B, P, true, true, false, false, CST>(cg, dl, len, MASK{}, rsbits, cvl, rs0, yl, 0, st);
                else
                    sweep<ORDER, ADJ, B, P, true, true, false, false, false>(cg, dl, len, MASK{}, MASK{}, nullptr, 0, yl, 0, st);
#pragma unroll
                for (int b = 0; b < B; ++b)
#pragma unroll
                    for (int q = 0; q < 3; ++q) v[b][q] = L::get(st[b / W][q], b % W);
#pragma unroll
                for (int k = 0; k < M; ++k) Pm[k] = Pc[k];
                warp_scan<ORDER, false, B, P>(Pm, v, lane);
                // ---- B: causal from the true entering state, in place
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        float w[W];
#pragma unroll
                        for (int h = 0; h < W; ++h) w[h] = v[u * W + h][q];
                        st[u][q] = L::make(w);
                    }
                if (cst) {
                    sweep<ORDER, ADJ, B, P, true, false, true, true, CST>(cg, dl, len, rebits, rsbits, cvl, rs0, yl, rank0, st);
                    apply_line_tails<ORDER, ADJ, B, P, CST>(ml, yl, line_re, lane, cvl);
                } else if (maps) {
                    sweep<ORDER, ADJ, B, P, true, false, true, true, false>(cg, dl, len, rebits, MASK{}, nullptr, 0, yl, rank0, st);
                    apply_line_tails<ORDER, ADJ, B, P, false>(ml, yl, line_re, lane, nullptr);
                } else {
                    sweep<ORDER, ADJ, B, P, true, false, true, false, false>(cg, dl, len, rebits, MASK{}, nullptr, 0, yl, rank0, st);
                }
                // ---- C: anticausal from zero at the chunk end
#pragma unroll
                for (int u = 0; u < U; ++u) st[u][0] = st[u][1] = st[u][2] = L::zero();
                if (cst) sweep<ORDER, ADJ, B, P, false, false, false, true, CST>(cg, dl, len, rebits, MASK{}, cvl, 0, yl, rank0 + nre - 1, st);
                else if (maps) sweep<ORDER, ADJ, B, P, false, false, false, true, false>(cg, dl, len, rebits, MASK{}, nullptr, 0, yl, rank0 + nre - 1, st);
                else sweep<ORDER, ADJ, B, P, false, false, false, false, false>(cg, dl, len, rebits, MASK{}, nullptr, 0, yl, 0, st);
#pragma unroll
                for (int b = 0; b < B; ++b)
#pragma unroll
                    for (int q = 0; q < 3; ++q) v[b][q] = L::get(st[b / W][q], b % W);
#pragma unroll
                for (int k = 0; k < M; ++k) Pm[k] = Pa[k];
                warp_scan<ORDER, true, B, P>(Pm, v, lane);
                // ---- D: anticausal from the true entering state, in place
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        float w[W];
#pragma unroll
                        for (int h = 0; h < W; ++h) w[h] = v[u * W + h][q];
                        st[u][q] = L::make(w);
                    }
                if (cst) sweep<ORDER, ADJ, B, P, false, false, true, true, CST>(cg, dl, len, rebits, rsbits, cvl, rs0 + nrs - 1, yl, rank0 + nre - 1, st);
                else if (maps) sweep<ORDER, ADJ, B, P, false, false, true, true, false>(cg, dl, len, rebits, MASK{}, nullptr, 0, yl, rank0 + nre - 1, st);
                else sweep<ORDER, ADJ, B, P, false, false, true, false, false>(cg, dl, len, rebits, MASK{}, nullptr, 0, yl, 0, st);
                __syncwarp();
            }
        };
        if (active) {
            if (C <= 64) filter(Bits64{rebits.lo}, Bits64{rsbits.lo});
            else filter(rebits, rsbits);
        }
        __syncthreads();
        // ---- store
        if (pv) {
            for (int u = 0; u < (nb + 1) / 2; ++u) {
                float *d0 = a.out + slice_of(gi, 2 * u) * a.plane;
                float *d1 = 2 * u + 1 < nb ? a.out + slice_of(gi, 2 * u + 1) * a.plane : nullptr;
                const float *db = ds + (int64_t)buf * B * R * ss + (int64_t)u * 2 * R * ss;
                for (int r = 0; r < lines_here; ++r) {
                    float4 *g0 = reinterpret_cast<float4 *>(d0 + (line0 + r) * a.line_stride);
                    float4 *g1 = d1 ? reinterpret_cast<float4 *>(d1 + (line0 + r) * a.line_stride) : nullptr;
                    const float4 *sr = reinterpret_cast<const float4 *>(db + 2 * r * ss);
#pragma unroll 4
                    for (int q = threadIdx.x; q < n / 4; q += blockDim.x) {
                        const float4 y0 = sr[2 * q], y1 = sr[2 * q + 1];
                        g0[q] = make_float4(y0.x, y0.z, y1.x, y1.z);
                        if (g1) g1[q] = make_float4(y0.y, y0.w, y1.y, y1.w);
                    }
                }
            }
        }
        if (svy && 4 * cq < lines_here) {
            for (int u = 0; u < (nb + 1) / 2; ++u) {
                float *d0 = a.out + slice_of(gi, 2 * u) * a.plane + line0 + 4 * cq;
                float *d1 = 2 * u + 1 < nb ? a.out + slice_of(gi, 2 * u + 1) * a.plane + line0 + 4 * cq
                                           : nullptr;
                const T *db = dt + ((int64_t)buf * U * R + (int64_t)u * R + 4 * cq) * ss;
#pragma unroll 4
                for (int k = yk1; k < n; k += ykstep) {
                    float y0[4], y1[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const T v = db[i * ss + k];
                        y0[i] = L::get(v, 0);
                        y1[i] = L::get(v, 1);
                    }
                    *reinterpret_cast<float4 *>(d0 + (int64_t)k * a.pt_stride) =
                        make_float4(y0[0], y0[1], y0[2], y0[3]);
                    if (d1)
                        *reinterpret_cast<float4 *>(d1 + (int64_t)k * a.pt_stride) =
                            make_float4(y1[0], y1[1], y1[2], y1[3]);
                }
            }
        }
        for (int b = 0; b < (pv || svy ? 0 : nb); ++b) {
            float *dst = a.out + slice_of(gi, b) * a.plane;
            const float *db = ds + (int64_t)buf * B * R * ss + (b / W) * W * R * ss + b % W;
            if (a.pt_stride == 1) {
                for (int r = 0; r < lines_here; ++r) {
                    float *g = dst + (line0 + r) * a.line_stride;
                    const float *s = db + W * r * ss;
                    if (vec) {
                        for (int q = threadIdx.x; q < n / 4; q += blockDim.x)
                            reinterpret_cast<float4 *>(g)[q] = reinterpret_cast<const float4 *>(s)[q];
                    } else {
                        for (int k = threadIdx.x; k < n; k += blockDim.x) g[k] = s[W * k];
                    }
                }
            } else if (yr < lines_here) {
                float *g = dst + (line0 + yr) + (int64_t)yk0 * a.pt_stride;
                const float *s = db + W * yr * ss;
                for (int k = yk0; k < n; k += P, g += row_step) *g = s[W * k];
            }
        }
        if (!dbl) __syncthreads();   // stores read the buffer the next copies fill
    }
    cp_async_wait_all();   // a CTA without slices still owns its map copies
}

template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
__global__ void __launch_bounds__(R * P) tile_kernel(TileArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_body<ORDER, ADJ, R, B, P, CST>(a, blockIdx.x, blockIdx.y, gridDim.y, smem_raw);
}

// The constant-extension kernels are compiled for a number of resident CTAs:
// two for 256 threads (128 registers a thread; their adjoint needs about 170
// and would otherwise run one CTA per SM), else about 170 registers, what
// they use anyway.
template <int R, int P>
constexpr int kCstMinCtas = R * P >= 256 ? 2 : 65536 / (R * P * 168);

template <int ORDER, bool ADJ, int R, int B, int P>
__global__ void __launch_bounds__(R * P, (kCstMinCtas<R, P>)) tile_kernel_cst(TileArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_body<ORDER, ADJ, R, B, P, true>(a, blockIdx.x, blockIdx.y, gridDim.y, smem_raw);
}

// Several domains in one launch.  The work list holds, domain after domain,
// one item per (line block, CTA row) of that domain's own grid: item i of
// domain d is line block i % gx[d] and row i / gx[d] of rows[d].  Persistent
// CTAs take items from a queue counter (zeroed by the host before the
// launch) until the list is exhausted, so ragged domains share the GPU
// without a tail per domain.
constexpr int kMaxMulti = 32;
struct MultiArgs {
    TileArgs dom[kMaxMulti];
    int64_t first[kMaxMulti + 1];   // first item of each domain; first[ndom] = total
    int64_t gx[kMaxMulti];          // line blocks per domain
    int64_t rows[kMaxMulti];        // CTA rows per domain
    unsigned long long *queue;      // item counter
    int ndom;
};

template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
__device__ __forceinline__ void multi_body(const MultiArgs &m, unsigned char *smem_raw);

template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
__global__ void __launch_bounds__(R * P) tile_multi_kernel(const __grid_constant__ MultiArgs m)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    multi_body<ORDER, ADJ, R, B, P, CST>(m, smem_raw);
}

template <int ORDER, bool ADJ, int R, int B, int P>
__global__ void __launch_bounds__(R * P, (kCstMinCtas<R, P>))
    tile_multi_kernel_cst(const __grid_constant__ MultiArgs m)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    multi_body<ORDER, ADJ, R, B, P, true>(m, smem_raw);
}

template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
__device__ __forceinline__ void multi_body(const MultiArgs &m, unsigned char *smem_raw)
{
    __shared__ long long item_s;
    const int64_t total = m.first[m.ndom];
    for (;;) {
        __syncthreads();   // the previous item is done with shared memory
        if (threadIdx.x == 0) item_s = (long long)atomicAdd(m.queue, 1ull);
        __syncthreads();
        const int64_t item = item_s;
        if (item >= total) break;
        int d = 0;
        while (d + 1 < m.ndom && m.first[d + 1] <= item) ++d;
        const int64_t i = item - m.first[d];
        tile_body<ORDER, ADJ, R, B, P, CST>(m.dom[d], i % m.gx[d], i / m.gx[d], m.rows[d], smem_raw);
    }
}

}  // namespace rfvh
