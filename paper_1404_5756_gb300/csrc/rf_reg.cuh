// rf_reg.cuh -- register-resident filter kernel (the default path for lines
// of up to 32 chunks of at most 32 points and 2-D coefficients).
//
// Each thread owns one chunk of C consecutive points of one line for four
// slices (levels or variables sharing the line's coefficients), held in
// registers as two pairs of FP32 values (fma/add/mul .f32x2: one instruction
// advances two slices).  The P lanes of a line sit in one warp (32/P lines
// per warp).  Lines move between global memory and the registers through a
// padded shared-memory transpose with coalesced global accesses; the sweeps
// themselves touch no shared memory except the per-point coefficients read
// through L1.  Per line and slice group, for each of the K iterations:
//   A  causal sweep of every chunk from zero state -> chunk end state
//   scan of (Phi_chunk, end state) over the P lanes (warp shuffles)
//   B  causal sweep from the true entering state, in place, recording the
//      state at every segment end
//   tails: the recorded states become the anticausal start states through
//      the FP64-built coastal maps (compensated FP32)
//   C  anticausal sweep of every chunk from zero state (start states
//      injected at the segment ends) -> chunk end state
//   reverse scan
//   D  anticausal sweep from the true entering state, in place
// The adjoint runs the same schedule with the transposed steps: A/B are the
// transposed anticausal pass (run left to right), C/D the transposed causal
// pass, and the coastal maps are applied transposed.
//
// Land carries the coefficients (0, 0, 0, -1) and steps with the reset factor
// g = 0 (1 at sea), so one land step maps any state to zero and outputs
// zero; g comes from the chunk's land bits.  The only per-point events are
// the segment ends (bit masks per chunk): B records the state after each,
// and the anticausal-direction sweeps C and D start each segment from its
// start state there.  Land inputs are zeroed when the chunk is loaded.
#pragma once
#include <cstdint>

#include "rf_steps.cuh"

namespace rfvh {

typedef unsigned long long u64;

// Per (line, lane) record of the register kernel: the chunk's segment events
// and land points (bit k <-> point k of the chunk; points past the line's
// end count as land), and the number of segment ends on the line before it.
struct RegLane {
    u64 ends;
    u64 starts;
    u64 land;
    int rank0;
    int nre;
};

// Transfer matrices per (line, lane): forward causal, forward anticausal,
// adjoint causal, adjoint anticausal (9 floats each, row-major, acting on the
// delta state; 1 float each for order 1).
template <int ORDER>
struct RXF {
    static constexpr int mat = ORDER == 3 ? 9 : 1;
    static constexpr int size = 4 * mat;
};

struct RegArgs {
    const float *in;          // field of this domain, [nvar][nz][ny][nx]
    float *out;
    const float4 *coef;       // [nlines][C][P] (beta, -e, -c1, -c2); land = 0
    const RegLane *lanes;     // [nlines][P]
    const float *xfer;        // [nlines][P][RXF::size]
    const int32_t *tail_base; // [nlines + 1] first coastal map of each line
    const float2 *tmap;       // [ntail][9] hi/lo pairs, consecutive along each line
    int64_t n, nlines;        // line length, lines per slice
    int64_t nx;               // grid row length (x pass: = n; y pass: column stride)
    int64_t plane;            // floats per slice
    int64_t nz, k0, nk;       // slices of this launch: (s / nk) * nz + k0 + s % nk
    int64_t nslices;          // nvar * nk
    int64_t ngroups;          // ceil(nslices / (2 * pairs per thread))
    int max_re;               // record slots per line (>= most segment ends on a line)
    int vec4;                 // 16-byte staging allowed (aligned base, nx % 4 == 0)
    int iters;
    int zero;                 // always 0; offsets the sweeps' coefficient pointers so the
                              // compiler cannot merge their loads (which would keep every
                              // coefficient of the chunk in registers across the sweeps)
    unsigned *status;         // device status word: bit 0 set if a bounded wait gave up
    int wait_polls;           // bound of the coefficient copy's wait (polls; 0: give up at once)
    // carried coasts (1st-RF, CARRY kernels): per segment [2][kc - 1] (mu at
    // its end, lambda at its start) of this direction, in boundary-map order
    const float *carry;
    int kc;                   // K
    int rs;                   // 64-bit record values per (segment, pair): NS, or 2 + 2 kc
};

// Record of one (segment, pair) in the carried-coast kernels: [0] the state
// recorded at the segment's end, then its start state M X + sum mu X; [1]
// the state entering the segment; [2, 2 + kc) the end's states of the
// iterations; [2 + kc, 2 + 2 kc) the start's states.
constexpr int kRecEnter = 1, kRecX = 2;

// Shared-memory layout of the register kernel (bytes):
//   16 bytes: the mbarrier of the coefficient copy;
//   the CTA's coefficient block: LC lines x C x P float4 (LC = 32/P lines for
//     the x pass, R = NW 32/P for the y pass), copied by one bulk copy;
//   staging of the four slices of a group:
//     x pass: per warp 4 slices x (32/P lines x P chunks x (C + 4) floats),
//     y pass: for the CTA 4 slices x R columns x pitch floats,
//             pitch = P (C + 4) + 4;
//   per warp the segment-end records: 32/P lines x slots x 2 NS 64-bit
//     values (the (co)state of both pairs at one segment end).
__host__ __device__ constexpr int reg_pitch(int C, int P) { return P * (C + 4) + 4; }

__host__ __device__ inline int64_t reg_coef_bytes(int dir, int C, int P, int NW)
{
    const int LC = dir == 0 ? 32 / P : NW * (32 / P);
    return (int64_t)LC * C * P * 16;
}

__host__ __device__ inline int64_t reg_stage_bytes(int dir, int C, int P, int NW, int npr)
{
    const int LPW = 32 / P, SG = 2 * npr;
    return dir == 0 ? (int64_t)NW * SG * LPW * P * (C + 4) * 4
                    : (int64_t)SG * NW * LPW * reg_pitch(C, P) * 4;
}

// rs: 64-bit record values per (segment, pair) (0: the state size NS).
__host__ __device__ inline int64_t reg_smem_bytes(int dir, int order, int C, int P, int NW,
                                                  int max_re, int npr, int rs = 0)
{
    const int LPW = 32 / P, NS = rs > 0 ? rs : order == 3 ? 3 : 1;
    const int64_t rec = (int64_t)NW * LPW * (max_re > 0 ? max_re : 1) * npr * NS * 8;
    return 16 + reg_coef_bytes(dir, C, P, NW) + reg_stage_bytes(dir, C, P, NW, npr) + rec;
}

// ---------------------------------------------------------------- bulk copy
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// One bulk copy global -> this CTA's shared memory, completing on mbarrier
// bar (both addresses and the size multiples of 16 bytes).
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Bounded wait for phase 0 of bar: true once the copy has landed, false if
// it has not after `tries` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, int tries)
{
    for (int i = 0; i < tries; ++i) {
        unsigned ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(smem_u32(bar)) : "memory");
        if (ok) return true;
    }
    return false;
}

// ---------------------------------------------------------------- steps
// Forward step, state (p, d1, d2) of the delta form; g = 1 at sea, 0 at land
// (land carries the coefficients (0, 0, 0, -1), so one step maps any state
// to zero and outputs zero).
template <int ORDER>
__device__ __forceinline__ u64 rstep_f(u64 x, u64 b, u64 ne, u64 nc1, u64 nc2, u64 g, u64 *s)
{
    if (ORDER == 3) {
        u64 t = V2::mul(b, x);
        t = V2::fma(nc2, s[2], t);
        t = V2::fma(nc1, s[1], t);
        t = V2::fma(ne, s[0], t);
        s[2] = V2::add(s[2], t);
        s[1] = V2::fma(g, s[1], s[2]);
        s[0] = V2::fma(g, s[0], s[1]);
        return s[0];
    }
    const u64 t = V2::fma(ne, s[0], V2::mul(b, x));
    s[0] = V2::fma(g, s[0], t);
    return s[0];
}

// Transposed step: costate (l0, l1, l2) of (p, d1, d2), input y: the exact
// transpose of the forward step written as the reversed sequence of its
// elementary operations (the same land values zero it).
template <int ORDER>
__device__ __forceinline__ u64 rstep_a(u64 y, u64 b, u64 ne, u64 nc1, u64 nc2, u64 g, u64 *s)
{
    if (ORDER == 3) {
        s[0] = V2::fma(g, s[0], y);
        s[1] = V2::fma(g, s[1], s[0]);
        s[2] = V2::fma(g, s[2], s[1]);
        const u64 out = V2::mul(b, s[2]);
        s[0] = V2::fma(ne, s[2], s[0]);
        s[1] = V2::fma(nc1, s[2], s[1]);
        s[2] = V2::fma(nc2, s[2], s[2]);
        return out;
    }
    s[0] = V2::fma(g, s[0], y);
    const u64 out = V2::mul(b, s[0]);
    s[0] = V2::fma(ne, s[0], s[0]);
    return out;
}

// ---------------------------------------------------------------- sweeps
// One sweep over the thread's chunk for both pairs.  CAUSAL walks up.  WRITE
// stores the outputs in place.  REC (causal direction): record the state
// after each segment end into rec[slot].  Anticausal direction: the state is
// set from rec[slot] before a segment end is stepped.  slot counts segment
// ends on the line: from rank0 up (causal) or down from rank0 + nre - 1
// (anticausal).  Land (bit set in `land`) steps with g = 0.  CARRY (carried
// coasts, first order; records of RS values): the causal sweeps set the state
// from rec[slot][kRecEnter] before a segment start is stepped, and the
// anticausal WRITE sweep records the state after each segment start into
// rec[slot][soff].
template <int ORDER, bool ADJ, bool CAUSAL, bool WRITE, bool REC, int C, int P, int NPR,
          bool CARRY = false>
__device__ __forceinline__ void rsweep(u64 (&x)[NPR][C], u64 (&st)[NPR][3],
                                       const float4 *__restrict__ cp, u64 ends, u64 land,
                                       u64 *__restrict__ rec, int slot, u64 starts = 0ull,
                                       int RS = ORDER == 3 ? 3 : 1, int soff = 0)
{
    constexpr int NS = ORDER == 3 ? 3 : 1;
    if (!CARRY) RS = NS;
    const u64 one = V2::bc(1.f);
#pragma unroll
    for (int kk = 0; kk < C; ++kk) {
        const int k = CAUSAL ? kk : C - 1 - kk;
        const float4 c = cp[k * P];
        const u64 b = V2::bc(c.x), ne = V2::bc(c.y);
        const u64 nc1 = ORDER == 3 ? V2::bc(c.z) : 0ull, nc2 = ORDER == 3 ? V2::bc(c.w) : 0ull;
        const u64 g = ((land >> k) & 1ull) ? 0ull : one;
        const bool at_end = (ends >> k) & 1ull;
        if (!CAUSAL && at_end) {
#pragma unroll
            for (int p = 0; p < NPR; ++p)
#pragma unroll
                for (int q = 0; q < NS; ++q) st[p][q] = rec[(slot * NPR + p) * RS + q];
            --slot;
        }
        if (CARRY && CAUSAL && ((starts >> k) & 1ull)) {
#pragma unroll
            for (int p = 0; p < NPR; ++p) st[p][0] = rec[(slot * NPR + p) * RS + kRecEnter];
        }
#pragma unroll
        for (int p = 0; p < NPR; ++p) {
            const u64 y = ADJ ? rstep_a<ORDER>(x[p][k], b, ne, nc1, nc2, g, st[p])
                              : rstep_f<ORDER>(x[p][k], b, ne, nc1, nc2, g, st[p]);
            if (WRITE) x[p][k] = y;
        }
        if (CARRY && !CAUSAL && WRITE && ((starts >> k) & 1ull)) {
            // slot + 1 is the segment of this start (its end is passed)
#pragma unroll
            for (int p = 0; p < NPR; ++p) rec[((slot + 1) * NPR + p) * RS + soff] = st[p][0];
        }
        if (CAUSAL && (REC || CARRY) && at_end) {
            if (REC) {
#pragma unroll
                for (int p = 0; p < NPR; ++p)
#pragma unroll
                    for (int q = 0; q < NS; ++q) rec[(slot * NPR + p) * RS + q] = st[p][q];
            }
            ++slot;
        }
    }
}

// Exclusive scan of affine chunk maps over the P lanes of a line (lane
// groups of width P in the warp).  Lane l holds x -> Pm x + v; afterwards v
// is the state entering its chunk (forward: from lanes 0..l-1; REV: from
// lanes P-1..l+1).  Pm is consumed.
template <int ORDER, bool REV, int P, int NPR>
__device__ __forceinline__ void rscan(float *Pm, u64 (&v)[NPR][3], int l)
{
    constexpr int M = RXF<ORDER>::mat, NS = ORDER == 3 ? 3 : 1;
#pragma unroll
    for (int d = 1; d < P; d <<= 1) {
        float Pn[M];
        u64 vn[NPR][NS];
#pragma unroll
        for (int k = 0; k < M; ++k)
            Pn[k] = REV ? __shfl_down_sync(0xffffffffu, Pm[k], d, P)
                        : __shfl_up_sync(0xffffffffu, Pm[k], d, P);
#pragma unroll
        for (int p = 0; p < NPR; ++p)
#pragma unroll
            for (int q = 0; q < NS; ++q)
                vn[p][q] = REV ? __shfl_down_sync(0xffffffffu, v[p][q], d, P)
                               : __shfl_up_sync(0xffffffffu, v[p][q], d, P);
        const bool take = REV ? (l + d < P) : (l >= d);
        if (take) {
            if (ORDER == 3) {
                u64 m[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) m[k] = V2::bc(Pm[k]);
#pragma unroll
                for (int p = 0; p < NPR; ++p) {
                    u64 nv[3];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        nv[r] = V2::fma(m[3 * r], vn[p][0],
                                        V2::fma(m[3 * r + 1], vn[p][1],
                                                V2::fma(m[3 * r + 2], vn[p][2], v[p][r])));
#pragma unroll
                    for (int r = 0; r < 3; ++r) v[p][r] = nv[r];
                }
                if (2 * d < P) {
                    float o[9];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            o[3 * r + c] = fmaf(Pm[3 * r], Pn[c],
                                                fmaf(Pm[3 * r + 1], Pn[3 + c], Pm[3 * r + 2] * Pn[6 + c]));
#pragma unroll
                    for (int k = 0; k < 9; ++k) Pm[k] = o[k];
                }
            } else {
                const u64 m = V2::bc(Pm[0]);
#pragma unroll
                for (int p = 0; p < NPR; ++p) v[p][0] = V2::fma(m, vn[p][0], v[p][0]);
                if (2 * d < P) Pm[0] *= Pn[0];
            }
        }
    }
#pragma unroll
    for (int p = 0; p < NPR; ++p)
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const u64 t = REV ? __shfl_down_sync(0xffffffffu, v[p][q], 1, P)
                              : __shfl_up_sync(0xffffffffu, v[p][q], 1, P);
            v[p][q] = (REV ? l == P - 1 : l == 0) ? 0ull : t;
        }
}

// Coastal maps of one line: each of its P lanes takes segment ends
// q = l, l + P, ...; the recorded state of each slice becomes M X (adjoint
// M^T X), applied in compensated FP32 (rf_steps.cuh).  Without imaginary
// points (ml null) every start state is zero.
// CARRY (carried coasts, iteration it, records of RS values, mu the line's
// history weights, kc - 1 per segment): the recorded state is also kept as
// the iteration's X, and the start state gains sum_d mu_d X_{it-d}.
template <int ORDER, bool ADJ, int P, int NPR, bool CARRY = false>
__device__ __forceinline__ void rtails(u64 *__restrict__ rec, const float2 *__restrict__ ml,
                                       int nre_line, int l, int RS = ORDER == 3 ? 3 : 1,
                                       const float *__restrict__ mu = nullptr, int it = 0,
                                       int kc = 1)
{
    constexpr int NS = ORDER == 3 ? 3 : 1;
    if (!CARRY) RS = NS;
    for (int q = l; q < nre_line; q += P) {
        u64 *r = rec + q * NPR * RS;
        if (!ml) {
#pragma unroll
            for (int p = 0; p < NPR; ++p)
#pragma unroll
                for (int k = 0; k < NS; ++k) r[p * RS + k] = 0ull;
            continue;
        }
#pragma unroll
        for (int p = 0; p < NPR; ++p) {
            if (CARRY) r[p * RS + kRecX + it] = r[p * RS];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float X[3] = {0.f, 0.f, 0.f}, Y[3];
#pragma unroll
                for (int k = 0; k < NS; ++k) X[k] = V2::get(r[p * RS + k], h);
                apply_tail<ORDER, ADJ>(ml + 9 * q, X, Y);
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    float lo = V2::get(r[p * RS + k], 0), hi = V2::get(r[p * RS + k], 1);
                    if (h == 0) lo = Y[k];
                    else hi = Y[k];
                    r[p * RS + k] = V2::pack(lo, hi);
                }
            }
            if (CARRY) {
                const float *m = mu + (int64_t)q * 2 * (kc - 1);
                u64 y = r[p * RS];
                for (int d = 1; d <= it; ++d)
                    y = V2::fma(V2::bc(m[d - 1]), r[p * RS + kRecX + it - d], y);
                r[p * RS] = y;
            }
        }
    }
}

// Carried coasts: the state entering each segment of the line in iteration
// it + 1, sum_{d=1..it+1} lambda_d S_{it+1-d} (lam: the line's weights).
template <int P, int NPR>
__device__ __forceinline__ void rheads(u64 *__restrict__ rec, const float *__restrict__ lam,
                                       int nre_line, int l, int RS, int it, int kc)
{
    for (int q = l; q < nre_line; q += P) {
        u64 *r = rec + q * NPR * RS;
        const float *w = lam + (int64_t)q * 2 * (kc - 1) + (kc - 1);
#pragma unroll
        for (int p = 0; p < NPR; ++p) {
            u64 h = 0ull;
            for (int d = 1; d <= it + 1; ++d)
                h = V2::fma(V2::bc(w[d - 1]), r[p * RS + kRecX + kc + it + 1 - d], h);
            r[p * RS + kRecEnter] = h;
        }
    }
}


// Plane index of slice s of a launch.
__device__ __forceinline__ int64_t reg_plane(const RegArgs &a, int64_t s)
{
    return (s / a.nk) * a.nz + a.k0 + s % a.nk;
}

// Pack chunk values of two slices (u from slice 2p, w from 2p+1) into
// pairs, zeroing land points, points past the line's end and missing slices.
template <int C>
__device__ __forceinline__ void reg_pack(u64 (&xp)[C], const float *c0, const float *c1,
                                         u64 land, bool ok0, bool ok1)
{
#pragma unroll
    for (int m = 0; m < C / 4; ++m) {
        const float4 u = *reinterpret_cast<const float4 *>(c0 + 4 * m);
        const float4 w = *reinterpret_cast<const float4 *>(c1 + 4 * m);
        const float uu[4] = {u.x, u.y, u.z, u.w}, ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool z = (land >> (4 * m + i)) & 1ull;
            xp[4 * m + i] = V2::pack(z || !ok0 ? 0.f : uu[i], z || !ok1 ? 0.f : ww[i]);
        }
    }
}

template <int C>
__device__ __forceinline__ void reg_unpack(const u64 (&xp)[C], float *c0, float *c1)
{
#pragma unroll
    for (int m = 0; m < C / 4; ++m) {
        float4 u, w;
        u.x = V2::get(xp[4 * m + 0], 0); w.x = V2::get(xp[4 * m + 0], 1);
        u.y = V2::get(xp[4 * m + 1], 0); w.y = V2::get(xp[4 * m + 1], 1);
        u.z = V2::get(xp[4 * m + 2], 0); w.z = V2::get(xp[4 * m + 2], 1);
        u.w = V2::get(xp[4 * m + 3], 0); w.w = V2::get(xp[4 * m + 3], 1);
        *reinterpret_cast<float4 *>(c0 + 4 * m) = u;
        *reinterpret_cast<float4 *>(c1 + 4 * m) = w;
    }
}

// Bound of the polls of the coefficient copy's mbarrier (each poll may
// suspend the thread for a while); far above any real copy time.  The
// plan's wait limit (rf_plan_set_wait_limit) bounds the first wait; after
// a wait gave up, the drain of the copy in flight uses this bound.
constexpr int kRegWaitTries = 1 << 20;

// ---------------------------------------------------------------- kernel
// DIR 0 (x pass): the CTA covers 32/P rows (blockIdx.x); its warps take
//   slice groups blockIdx.y * NW + warp, each staging its rows alone.
// DIR 1 (y pass): the CTA covers R = NW * 32/P adjacent columns
//   (blockIdx.x) and slice group blockIdx.y; the CTA stages the columns'
//   tile together.
// Both: the CTA's coefficient block arrives by one bulk copy while the data
// loads are in flight.
// The work of one CTA of one domain's grid (reg_grid): (blockIdx.x,
// blockIdx.y), or (bx_, by_) in a multi-domain launch (MULTI).
template <int ORDER, bool ADJ, int DIR, int C, int P, int NW, int NPR, bool CARRY, bool MULTI>
__device__ __forceinline__ void reg_body(const RegArgs &a, const unsigned bx_, const unsigned by_)
{
    // (the single-domain kernel reads the block index where it is used, so
    // no register holds it across the sweeps)
#define bx (MULTI ? bx_ : blockIdx.x)
#define by (MULTI ? by_ : blockIdx.y)
    constexpr int NS = ORDER == 3 ? 3 : 1, MX = RXF<ORDER>::mat;
    static_assert(!CARRY || ORDER == 1, "carried coasts are a first-order option");
    const int RS = CARRY ? a.rs : NS;
    constexpr int LPW = 32 / P, R = NW * LPW, LC = DIR == 0 ? LPW : R;
    constexpr int STG = DIR == 0 ? LPW * P * (C + 4) : R * reg_pitch(C, P);   // floats per slice
    constexpr int PITCH = reg_pitch(C, P);
    constexpr int SG = 2 * NPR;   // slices per group
    static_assert(C % 4 == 0 && C <= 64, "chunk");
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem);
    float4 *scoef = reinterpret_cast<float4 *>(smem + 16);
    float *stage = reinterpret_cast<float *>(smem + 16 + reg_coef_bytes(DIR, C, P, NW));
    u64 *recs = reinterpret_cast<u64 *>(smem + 16 + reg_coef_bytes(DIR, C, P, NW) +
                                        reg_stage_bytes(DIR, C, P, NW, NPR));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ql = lane / P, l = lane % P;   // line within the warp, lane on the line
    const int64_t n = a.n;

    const int64_t cline0 = (int64_t)bx * LC;                   // first line of the CTA
    const int nvalid = (int)min((int64_t)LC, a.nlines - cline0);        // its lines in the grid
    const int64_t line0 = DIR == 0 ? cline0 : cline0 + warp * LPW;      // first line of the warp
    const int64_t g = DIR == 0 ? (int64_t)by * NW + warp : (int64_t)by;
    const bool active = g < a.ngroups;   // x pass: warps past the last group only join barriers
    const int64_t myline0 = line0 + ql;
    const bool line_ok = myline0 < a.nlines;
    const int64_t line = line_ok ? myline0 : a.nlines - 1;   // past the end: compute, never store
    u64 *rec = recs + ((int64_t)warp * LPW + ql) * (a.max_re > 0 ? a.max_re : 1) * NPR * RS;

    // coefficient block of the CTA's lines: one bulk copy
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        bulk_copy_g2s(scoef, a.coef + cline0 * C * P, (unsigned)nvalid * C * P * 16u, bar);

    const RegLane li = a.lanes[line * P + l];
    const float *xf = a.xfer + (line * P + l) * RXF<ORDER>::size + (ADJ ? 2 * MX : 0);
    // segment ends on the line: the last lane's rank plus its own count
    const int nre_line = __shfl_sync(0xffffffffu, li.rank0 + li.nre, P - 1, P);
    const float2 *ml = a.tmap ? a.tmap + 9 * (int64_t)a.tail_base[line] : nullptr;
    // carried coasts: the line's history weights (mu, lambda per segment)
    const float *cw = CARRY ? a.carry + (int64_t)a.tail_base[line] * 2 * (a.kc - 1) : nullptr;

    int64_t off[SG];
    bool sok[SG];
#pragma unroll
    for (int b = 0; b < SG; ++b) {
        const int64_t s = g * SG + b;
        sok[b] = active && s < a.nslices;
        off[b] = sok[b] ? reg_plane(a, s) * a.plane : 0;
    }

    // ------------------------------------------------------------ stage in
    // Every load of the item is issued before the first shared-memory store
    // (compile-time trip counts: P C >= n bounds the points of a line).
    if (DIR == 0) {
        // the warp's rows of all four slices: coalesced loads into
        // chunk-padded rows (chunk k of a row at k (C + 4))
        float *ws = stage + warp * SG * STG;
        if (a.vec4) {
            constexpr int NJ = C * P / 128;   // float4 per lane per row
            float4 v[SG][LPW][NJ];
#pragma unroll
            for (int b = 0; b < SG; ++b)
#pragma unroll
                for (int q = 0; q < LPW; ++q) {
                    const int64_t row = line0 + q;
                    const float4 *src = reinterpret_cast<const float4 *>(a.in + off[b] + row * a.nx);
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int e4 = lane + 32 * j;
                        if (sok[b] && row < a.nlines && e4 * 4 < n) v[b][q][j] = __ldg(src + e4);
                    }
                }
#pragma unroll
            for (int b = 0; b < SG; ++b)
#pragma unroll
                for (int q = 0; q < LPW; ++q)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int e = 4 * (lane + 32 * j);
                        if (sok[b] && line0 + q < a.nlines && e < n)
                            *reinterpret_cast<float4 *>(ws + b * STG + q * P * (C + 4) +
                                                        (e / C) * (C + 4) + e % C) = v[b][q][j];
                    }
        } else {
            constexpr int NJ = C * P / 32;   // floats per lane per row
            float v[SG][LPW][NJ];
#pragma unroll
            for (int b = 0; b < SG; ++b)
#pragma unroll
                for (int q = 0; q < LPW; ++q) {
                    const int64_t row = line0 + q;
                    const float *src = a.in + off[b] + row * a.nx;
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int e = lane + 32 * j;
                        if (sok[b] && row < a.nlines && e < n) v[b][q][j] = __ldg(src + e);
                    }
                }
#pragma unroll
            for (int b = 0; b < SG; ++b)
#pragma unroll
                for (int q = 0; q < LPW; ++q)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int e = lane + 32 * j;
                        if (sok[b] && line0 + q < a.nlines && e < n)
                            ws[b * STG + q * P * (C + 4) + (e / C) * (C + 4) + e % C] = v[b][q][j];
                    }
        }
    } else {
        // the CTA's columns of all four slices: rows of R floats, transposed
        // into chunk-padded columns of pitch PITCH
        if (a.vec4 && nvalid == R) {
            constexpr int F = R / 4;                              // float4 per row
            constexpr int NJ = (C * P * F + NW * 32 - 1) / (NW * 32);   // per thread per slice
            float4 v[SG][NJ];
#pragma unroll
            for (int b = 0; b < SG; ++b) {
                const float *src = a.in + off[b] + cline0;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int t = threadIdx.x + NW * 32 * j, jr = t / F, f = t % F;
                    if (sok[b] && jr < n) v[b][j] = __ldg(reinterpret_cast<const float4 *>(src + jr * a.nx) + f);
                }
            }
#pragma unroll
            for (int b = 0; b < SG; ++b) {
                float *tile = stage + b * STG;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int t = threadIdx.x + NW * 32 * j, jr = t / F, f = t % F;
                    if (sok[b] && jr < n) {
                        const int pos = (jr / C) * (C + 4) + jr % C;
                        tile[(4 * f + 0) * PITCH + pos] = v[b][j].x;
                        tile[(4 * f + 1) * PITCH + pos] = v[b][j].y;
                        tile[(4 * f + 2) * PITCH + pos] = v[b][j].z;
                        tile[(4 * f + 3) * PITCH + pos] = v[b][j].w;
                    }
                }
            }
        } else {
            constexpr int NJ = (C * P * R + NW * 32 - 1) / (NW * 32);
            float v[SG][NJ];
#pragma unroll
            for (int b = 0; b < SG; ++b) {
                const float *src = a.in + off[b] + cline0;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int t = threadIdx.x + NW * 32 * j, jr = t / R, c = t % R;
                    if (sok[b] && jr < n && c < nvalid) v[b][j] = __ldg(src + jr * a.nx + c);
                }
            }
#pragma unroll
            for (int b = 0; b < SG; ++b) {
                float *tile = stage + b * STG;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int t = threadIdx.x + NW * 32 * j, jr = t / R, c = t % R;
                    if (sok[b] && jr < n && c < nvalid)
                        tile[c * PITCH + (jr / C) * (C + 4) + jr % C] = v[b][j];
                }
            }
        }
    }
    // the coefficients must have landed in every thread's view; give up
    // (flag, drain the copy, leave) if they do not arrive
    if (!__syncthreads_and(mbar_wait(bar, a.wait_polls))) {
        if (threadIdx.x == 0) atomicOr(a.status, 1u);
        mbar_wait(bar, kRegWaitTries);
        return;
    }

    const float4 *cp = scoef + (int64_t)(line - cline0) * C * P + l;
    const float *c0 = DIR == 0 ? stage + warp * SG * STG + (ql * P + l) * (C + 4)
                               : stage + (warp * LPW + ql) * PITCH + l * (C + 4);
    u64 x[NPR][C];
    const u64 land = li.land | (line_ok ? 0ull : ~0ull);
#pragma unroll
    for (int p = 0; p < NPR; ++p)
        reg_pack<C>(x[p], c0 + 2 * p * STG, c0 + (2 * p + 1) * STG, land, sok[2 * p], sok[2 * p + 1]);

    // ------------------------------------------------------------ filter
    if (active) {
        if (CARRY) {
            // the first iteration enters every segment from zero
            for (int q = l; q < nre_line; q += P)
#pragma unroll
                for (int p = 0; p < NPR; ++p) rec[(q * NPR + p) * RS + kRecEnter] = 0ull;
            __syncwarp();
        }
        for (int it = 0; it < a.iters; ++it) {
            u64 st[NPR][3];
            float Pm[MX];
            // A: local causal-direction sweep
#pragma unroll
            for (int p = 0; p < NPR; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) st[p][q] = 0ull;
            rsweep<ORDER, ADJ, true, false, false, C, P, NPR, CARRY>(
                x, st, cp + a.zero, li.ends, li.land, rec, CARRY ? li.rank0 : 0, li.starts, RS);
#pragma unroll
            for (int k = 0; k < MX; ++k) Pm[k] = __ldg(xf + k);
            rscan<ORDER, false, P, NPR>(Pm, st, l);
            // B: from the true state, recording segment ends
            rsweep<ORDER, ADJ, true, true, true, C, P, NPR, CARRY>(
                x, st, cp + 2 * a.zero, li.ends, li.land, rec, li.rank0, li.starts, RS);
            __syncwarp();
            if (line_ok) rtails<ORDER, ADJ, P, NPR, CARRY>(rec, ml, nre_line, l, RS, cw, it, a.kc);
            __syncwarp();
            // C: local anticausal-direction sweep
#pragma unroll
            for (int p = 0; p < NPR; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) st[p][q] = 0ull;
            rsweep<ORDER, ADJ, false, false, false, C, P, NPR, CARRY>(
                x, st, cp + 3 * a.zero, li.ends, li.land, rec, li.rank0 + li.nre - 1, li.starts, RS);
#pragma unroll
            for (int k = 0; k < MX; ++k) Pm[k] = __ldg(xf + MX + k);
            rscan<ORDER, true, P, NPR>(Pm, st, l);
            // D: from the true state (carried coasts: recording segment starts)
            rsweep<ORDER, ADJ, false, true, false, C, P, NPR, CARRY>(
                x, st, cp + 4 * a.zero, li.ends, li.land, rec, li.rank0 + li.nre - 1, li.starts, RS,
                kRecX + a.kc + it);
            __syncwarp();   // the records are rewritten by the next iteration's B
            if (CARRY && it + 1 < a.iters) {
                if (line_ok) rheads<P, NPR>(rec, cw, nre_line, l, RS, it, a.kc);
                __syncwarp();
            }
        }
    }

    // ------------------------------------------------------------ stage out
    // (each thread reads and writes only its own chunks of the staging until
    // the barrier below)
    float *c0w = const_cast<float *>(c0);
#pragma unroll
    for (int p = 0; p < NPR; ++p) reg_unpack<C>(x[p], c0w + 2 * p * STG, c0w + (2 * p + 1) * STG);
    if (DIR == 0) {
        __syncwarp();
        const float *ws = stage + warp * SG * STG;
#pragma unroll
        for (int b = 0; b < SG; ++b)
            for (int q = 0; q < LPW; ++q) {
                const int64_t row = line0 + q;
                if (row >= a.nlines || !sok[b]) continue;
                float *dst = a.out + off[b] + row * a.nx;
                const float *sq = ws + b * STG + q * P * (C + 4);
                if (a.vec4) {
                    for (int64_t e4 = lane; e4 * 4 < n; e4 += 32) {
                        const int e = (int)e4 * 4;
                        reinterpret_cast<float4 *>(dst)[e4] =
                            *reinterpret_cast<const float4 *>(sq + (e / C) * (C + 4) + e % C);
                    }
                } else {
                    for (int e = lane; e < n; e += 32) dst[e] = sq[(e / C) * (C + 4) + e % C];
                }
            }
    } else {
        __syncthreads();
#pragma unroll
        for (int b = 0; b < SG; ++b) {
            if (!sok[b]) continue;   // block-uniform
            const float *tile = stage + b * STG;
            float *dst = a.out + off[b] + cline0;
            if (a.vec4 && nvalid == R) {
                constexpr int F = R / 4;
                for (int t = threadIdx.x; t < n * F; t += NW * 32) {
                    const int j = t / F, f = t % F;
                    const int pos = (j / C) * (C + 4) + j % C;
                    float4 v;
                    v.x = tile[(4 * f + 0) * PITCH + pos];
                    v.y = tile[(4 * f + 1) * PITCH + pos];
                    v.z = tile[(4 * f + 2) * PITCH + pos];
                    v.w = tile[(4 * f + 3) * PITCH + pos];
                    reinterpret_cast<float4 *>(dst + j * a.nx)[f] = v;
                }
            } else {
                for (int t = threadIdx.x; t < n * R; t += NW * 32) {
                    const int j = t / R, c = t % R;
                    if (c < nvalid) dst[j * a.nx + c] = tile[c * PITCH + (j / C) * (C + 4) + j % C];
                }
            }
        }
    }
}

#undef bx
#undef by

template <int ORDER, bool ADJ, int DIR, int C, int P, int NW, int NPR, bool CARRY = false>
__global__ void __launch_bounds__(NW * 32, NPR == 2 ? 2 : 3) reg_kernel(const RegArgs a)
{
    reg_body<ORDER, ADJ, DIR, C, P, NW, NPR, CARRY, false>(a, 0u, 0u);
}

// One launch over several domains of the same chunking (a ragged batch):
// the 1-D grid is the concatenation of the domains' grids; cta0[d] is the
// first CTA of domain d, gx[d] the x extent of its grid.
constexpr int kRegMulti = 64;
struct RegMulti {
    int nd;
    int gx[kRegMulti];
    int64_t cta0[kRegMulti + 1];
    RegArgs dom[kRegMulti];
};

template <int ORDER, bool ADJ, int DIR, int C, int P, int NW, int NPR, bool CARRY = false>
__global__ void __launch_bounds__(NW * 32, NPR == 2 ? 2 : 3)
    reg_multi_kernel(const __grid_constant__ RegMulti m)
{
    const int64_t b = blockIdx.x;
    int lo = 0, hi = m.nd - 1;   // the domain d with cta0[d] <= b < cta0[d + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m.cta0[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int64_t r = b - m.cta0[lo];
    reg_body<ORDER, ADJ, DIR, C, P, NW, NPR, CARRY, true>(m.dom[lo], (unsigned)(r % m.gx[lo]),
                                                          (unsigned)(r / m.gx[lo]));
}

}  // namespace rfvh
