// rf_plan.cu -- C ABI of the recursive-filter library: plan construction
// (validation, sea segments, FP64 coefficients, coastal boundary maps, chunk
// transfer matrices) and the apply entry points.  See include/rfvh.h for the
// contract of every call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <new>
#include <mutex>
#include <vector>

#include "rfvh.h"
#include "rf_coef.cuh"
#include "rf_launch.h"
#include "rf_line.cuh"
#include "rf_reg_launch.h"
#include "rf_stream_launch.h"
#include "rf_tile.cuh"

using namespace rfvh;

namespace {

// One sea segment of a line: length scale and imaginary points at its end
// (the boundary map) and at its start (constant-extension coasts).
struct TailSpec {
    float sigma;
    int n_img;
    float sigma_h;
    int n_h;
};

// How one direction of one domain is launched for a given slice count.
struct LaunchCfg {
    bool reg = false;      // register-resident kernel (rf_reg.cuh)
    bool strm = false;     // streaming column kernel (rf_stream.cuh)
    bool tile = false;     // tile kernel (else the long-line kernel, unless reg)
    TileShape sh{0, 0};
    size_t smem = 0;
    int occ = 0;           // resident CTAs per SM
    int nbuf = 1;          // data buffers in shared memory (1 or 2)
    int64_t groups = 1;    // CTA rows along the slices
};

struct CfgEntry {
    int64_t nvar, nk;   // variables, levels per launch
    bool adjoint;
    LaunchCfg cfg;
};

// Everything one direction (x: rows, y: columns) of one domain needs.
struct Dir {
    int dir = 0;                     // 0: x (rows), 1: y (columns)
    int64_t n = 0, nlines = 0;       // line length, lines per slice
    int64_t pt_stride = 0, line_stride = 0;
    int64_t C = 0;                   // chunk length of the tile kernel (odd)
    int R = 0;                       // lines per CTA; 0 = long-line kernel
    size_t smem = 0;
    float4 *coef = nullptr;          // [ncl][nlines][n]
    int32_t *tail_base = nullptr;    // [ncl*nlines + 1] first boundary map of each line
    float2 *tmap = nullptr;          // [ntail][9] hi/lo pairs, consecutive along each line
    float4 *cvec = nullptr;          // [ntail][2] (m, s) of constant-extension coasts
    bool cst = false;                // constant-extension coasts in force
    int kc = 0;                      // carried coasts: K (0: not in force)
    float *carry = nullptr;          // [2 fwd/adj][ntail][2 mu/lambda][K - 1] history weights
    int P = 32;                      // lanes per line of the tile kernel (32 or 16)
    float *xfer = nullptr;           // [ncl][nlines][P][XF]
    float4 *coef_il_base = nullptr;  // interleaved coefficients with guards
    float4 *coef_il = nullptr;       // [ncl][nlines][C][P] (tile kernel)
    LaneInfo *lanes = nullptr;       // [ncl][nlines][P]
    int64_t ntail = 0;
    int max_re = 0;                  // most segment ends on one line
    // register-resident kernel (2-D coefficients, zero-input coasts, lines
    // of at most 1024 points): its chunking and tables
    RegShape rsh{0, 0};              // C, P; P = 0 marks "not available"
    float4 *rcoef = nullptr;         // [nlines][C][P] (beta, -e, -c1, -c2), land 0
    RegLane *rlanes = nullptr;       // [nlines][P]
    float *rxfer = nullptr;          // [nlines][P][4 * (9 or 1)]
    int max_ends = 0;                // most segment ends on one line
    // streaming column kernel (third-order y pass, 2-D coefficients): the
    // coefficients row-major, [n][nlines]
    float4 *tcoef = nullptr;
    std::vector<CfgEntry> cfgs;      // launch shapes chosen so far
};

struct Domain {
    rf_grid g{};
    unsigned *status = nullptr;      // the plan's device status word (not owned)
    const int *wait_polls = nullptr; // the plan's wait bound (not owned)
    int64_t ncl = 1;                 // levels with distinct coefficients
    Dir d[2];                        // 0: x, 1: y
    float *tscr = nullptr;           // boundary-map start states
    int64_t tscr_floats = 0;
    float *stage = nullptr;          // host-API staging
    int64_t stage_floats = 0;
    std::vector<std::pair<int64_t, int64_t>> batch;   // tuned (nvar, levels per batch)
};

}  // namespace

namespace {
// Launch shape of one pass of the multi-domain launch for nvar variables,
// over the domains whose lines in that direction run with P lanes each.
struct MultiCfg {
    int64_t nvar;
    bool adjoint;
    int dir;
    int P;
    TileShape sh;
    size_t smem;
    int occ;
};
}  // namespace

struct rf_plan_ {
    rf_options opt{};
    std::vector<Domain> dom;
    int64_t bytes = 0;
    int64_t launches = 0;
    rf_status sticky = RF_OK;
    unsigned long long *queue = nullptr;   // work-list counter of multi-domain launches
    unsigned *dstatus = nullptr;           // device status word: bit 0 = a bounded wait gave up
    int wait_polls = kRegWaitTries;        // bound of the kernels' device-side waits
    cudaStream_t s_in = nullptr, s_out = nullptr;   // copy streams of the host-buffer apply
    cudaEvent_t ev_in = nullptr, ev_done = nullptr, ev_out = nullptr;
    std::vector<MultiCfg> mcfg;            // multi-domain launch shapes chosen so far
    std::vector<std::pair<int64_t, bool>> multi_pref;   // tuned: (nvar, use multi-domain launches)
};

namespace {

constexpr size_t kSmemTarget = 112 * 1024;   // two CTAs per SM
constexpr size_t kSmemMax = 227 * 1024;

template <class T>
rf_status dev_alloc(T **p, int64_t count, int64_t *bytes)
{
    *p = nullptr;
    if (count <= 0) return RF_OK;
    size_t nb = sizeof(T) * (size_t)count;
    if (cudaMalloc((void **)p, nb) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return RF_ENOMEM;
    }
    *bytes += (int64_t)nb;
    return RF_OK;
}

void free_domain(Domain &d)
{
    for (Dir &q : d.d) {
        cudaFree(q.coef);
        cudaFree(q.tail_base);
        cudaFree(q.tmap);
        cudaFree(q.cvec);
        cudaFree(q.tcoef);
        cudaFree(q.carry);
        cudaFree(q.xfer);
        cudaFree(q.coef_il_base);
        cudaFree(q.lanes);
        cudaFree(q.rcoef);
        cudaFree(q.rlanes);
        cudaFree(q.rxfer);
    }
    cudaFree(d.tscr);
    cudaFree(d.stage);
    d = Domain{};
}

void free_plan(rf_plan_ *p)
{
    for (auto &d : p->dom) free_domain(d);
    cudaFree(p->queue);
    p->queue = nullptr;
    cudaFree(p->dstatus);
    p->dstatus = nullptr;
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_done) cudaEventDestroy(p->ev_done);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
}

rf_status check_options(const rf_options &o)
{
    if (o.order != 1 && o.order != 3) return RF_EINVAL;
    if (o.iters < 1 || (o.order == 3 && o.iters != 1)) return RF_EINVAL;
    if (!(o.img_factor >= 0.0)) return RF_EINVAL;   // NaN or negative; +inf is allowed
    if (o.norm != RF_NORM_GAUSS_PEAK && o.norm != RF_NORM_UNIT_SUM) return RF_EINVAL;
    if ((o.flags & ~(RF_FLAG_Q_CORRECTED | RF_FLAG_COAST_CONSTANT | RF_FLAG_COAST_CARRIED)) != 0 ||
        o.chunk < 0 || o.tile < 0)
        return RF_EINVAL;
    if ((o.flags & RF_FLAG_COAST_CONSTANT) && (o.flags & RF_FLAG_COAST_CARRIED)) return RF_EINVAL;
    // the kernels derive chunk lengths and tile shapes from the line length
    // (the autotuner picks launch shapes); no override is built
    if (o.chunk != 0 || o.tile != 0) return RF_EUNSUPPORTED;
    if ((o.flags & RF_FLAG_Q_CORRECTED) && o.order != 3) return RF_EINVAL;
    // the infinite imaginary sea is built for zero-input coasts only
    if (std::isinf(o.img_factor) && (o.flags & RF_FLAG_COAST_CONSTANT)) return RF_EUNSUPPORTED;
    return RF_OK;
}

rf_status check_grid(const rf_grid &g)
{
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return RF_EINVAL;
    if (!(g.mask_nz == 1 || g.mask_nz == g.nz)) return RF_EINVAL;
    if (!(g.L_nz == 1 || g.L_nz == g.nz)) return RF_EINVAL;
    // nz bounds the y extent of the launch grids (one CTA row per level)
    if (g.nx > (1 << 30) || g.ny > (1 << 30) || g.nz > 65535) return RF_EINVAL;
    if (g.nx * g.ny > ((int64_t)1 << 40)) return RF_EINVAL;
    return RF_OK;
}

// Constant-extension coasts in force: the option, and imaginary points to
// carry the edge values.
bool plan_cst(const rf_plan_ *p)
{
    return (p->opt.flags & RF_FLAG_COAST_CONSTANT) && p->opt.img_factor > 0.0;
}

// Carried coasts in force: the option, the 1st-RF with more than one
// iteration, and imaginary points to carry values.
bool plan_carry(const rf_plan_ *p)
{
    return (p->opt.flags & RF_FLAG_COAST_CARRIED) && p->opt.order == 1 && p->opt.iters > 1 &&
           p->opt.img_factor > 0.0;
}

// Floats per segment-end record of the long-line kernel: the start state,
// plus the last input (forward) or the tail-vector term (adjoint) with
// constant coasts; with carried coasts the start state, the state entering
// the segment and the K boundary states of each end.
int rec_floats(const Dir &q)
{
    return q.kc > 0 ? 2 + 2 * q.kc : q.cst ? 4 : 3;
}

rf_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return RF_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? RF_ENOMEM : RF_ECUDA;
}

#define RF_TRY(expr)                      \
    do {                                  \
        rf_status _s = (expr);            \
        if (_s != RF_OK) return _s;       \
    } while (0)

// ------------------------------------------------------------------ set-up
// Per-point coefficients of one direction in line-major order, computed in
// FP64 and stored as FP32 (beta, -e, -c1, -c2); land -> (0, 0, 0, -1); the
// last sea point of a segment gets beta negated.
__global__ void coef_lines_kernel(int64_t ncl, int64_t nx, int64_t ny, int along_y,
                                  const uint8_t *__restrict__ mask, int64_t mask_nz,
                                  const float *__restrict__ L, int64_t L_nz, int order,
                                  int K, int norm, int qc, float4 *__restrict__ out)
{
    const int64_t plane = nx * ny;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= ncl * plane) return;
    const int64_t lev = idx / plane, r = idx - lev * plane;
    const int64_t n = along_y ? ny : nx;
    const int64_t line = r / n, pos = r - line * n;
    const int64_t j = along_y ? pos : line, i = along_y ? line : pos;
    const uint8_t *m = mask + (mask_nz > 1 ? lev : 0) * plane;
    const int64_t p = j * nx + i;
    float4 c = make_float4(0.f, 0.f, 0.f, -1.f);
    if (m[p]) {
        const double s = (double)L[(L_nz > 1 ? lev : 0) * plane + p];
        const Coef64 k = coef_fp64(s, order, K, norm, qc != 0);
        c = make_float4((float)k.beta, -(float)k.e, -(float)k.c1, -(float)k.c2);
        const int64_t pn = along_y ? p + nx : p + 1;
        if (pos == n - 1 || !m[pn]) c.x = -c.x;
    }
    out[idx] = c;
}

// Boundary maps in FP64, stored as hi/lo FP32 pairs (hi = m rounded to
// FP32, lo = the rest rounded to FP32) for the compensated FP32 application;
// with constant-extension coasts (cvec non-null) also the segment's tail
// vector m (end) and head vector s (start), FP32.
__global__ void tail_kernel(int64_t n, const TailSpec *__restrict__ spec,
                            float2 *__restrict__ tmap, float4 *__restrict__ cvec, int order,
                            int K, int norm, int qc)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m[9];
    if (spec[i].n_img < 0)
        tail_map_inf_fp64((double)spec[i].sigma, order, K, norm, qc != 0, m);
    else
        tail_map_fp64((double)spec[i].sigma, spec[i].n_img, order, K, norm, qc != 0, m);
    for (int r = 0; r < 9; ++r) {
        const float hi = (float)m[r];
        tmap[9 * i + r] = make_float2(hi, (float)(m[r] - (double)hi));
    }
    if (cvec) {
        double h[3], t[3], unused[3];   // head at the start, tail at the end
        coast_vectors_fp64((double)spec[i].sigma, spec[i].n_img, order, K, norm, qc != 0, unused, t);
        coast_vectors_fp64((double)spec[i].sigma_h, spec[i].n_h, order, K, norm, qc != 0, h, unused);
        cvec[2 * i] = make_float4((float)t[0], (float)t[1], (float)t[2], 0.f);
        cvec[2 * i + 1] = make_float4((float)h[0], (float)h[1], (float)h[2], 0.f);
    }
}

// One-step matrix of the delta form with the reset factor (rf_steps.cuh),
// from the stored FP32 coefficients.
__device__ void step_matrix(const float4 &cf, double *A, int order)
{
    const double b = fabs((double)cf.x), e = -cf.y, c1 = -cf.z, c2 = -cf.w;
    const double g = b != 0.0 ? 1.0 : 0.0;
    if (order == 1) {
        A[0] = g - e;
        return;
    }
    A[0] = g - e; A[1] = g - c1; A[2] = 1.0 - c2;
    A[3] = -e;    A[4] = g - c1; A[5] = 1.0 - c2;
    A[6] = -e;    A[7] = -c1;    A[8] = 1.0 - c2;
}

__device__ void mm3(const double *P, const double *Q, double *O)
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            O[3 * r + c] = P[3 * r] * Q[c] + P[3 * r + 1] * Q[3 + c] + P[3 * r + 2] * Q[6 + c];
}

// Lane-interleaved copy of one direction's coefficients for the tile kernel
// (step j of lane l of a line at [line][j][l], P lanes per line, points past
// the line's end are land), with the segment-end flags moved into per-lane
// bit masks and the rank of each lane's first segment end on its line; the
// same for the segment starts (a sea point after land or at the line's
// start).  P threads per line; a warp's lines past the end work on the last
// line (every lane joins the shuffles) and write nothing.
__global__ void interleave_kernel(int64_t nlines_total, int64_t n, int C, int P,
                                  const float4 *__restrict__ coef, float4 *__restrict__ il,
                                  LaneInfo *__restrict__ lanes)
{
    const int64_t line0 = blockIdx.x * (int64_t)(blockDim.x / P) + threadIdx.x / P;
    const int lane = threadIdx.x % P;
    if (blockIdx.x * (int64_t)(blockDim.x / P) + (threadIdx.x / 32) * (32 / P) >= nlines_total)
        return;   // whole warps past the end exit together
    const bool ok = line0 < nlines_total;
    const int64_t line = ok ? line0 : nlines_total - 1;
    const float4 *src = coef + line * n;
    float4 *dst = il + line * C * P + lane;
    unsigned long long bits[2] = {0ull, 0ull}, sbits[2] = {0ull, 0ull};
    for (int j = 0; j < C; ++j) {
        const int64_t k = (int64_t)lane * C + j;
        float4 c = k < n ? src[k] : make_float4(0.f, 0.f, 0.f, -1.f);
        if (c.x != 0.f && (k == 0 || src[k - 1].x == 0.f)) sbits[j >> 6] |= 1ull << (j & 63);
        if (__float_as_uint(c.x) >> 31) {
            bits[j >> 6] |= 1ull << (j & 63);
            c.x = fabsf(c.x);
        }
        if (ok) dst[(int64_t)j * P] = c;
    }
    const int nre = __popcll(bits[0]) + __popcll(bits[1]);
    const int nrs = __popcll(sbits[0]) + __popcll(sbits[1]);
    int incl = nre, incs = nrs;
    for (int d = 1; d < P; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d, P);
        const int u = __shfl_up_sync(0xffffffffu, incs, d, P);
        if (lane >= d) {
            incl += t;
            incs += u;
        }
    }
    LaneInfo li;
    li.re.lo = bits[0];
    li.re.hi = bits[1];
    li.rank0 = incl - nre;
    li.nre = nre;
    li.rs.lo = sbits[0];
    li.rs.hi = sbits[1];
    li.rs0 = incs - nrs;
    li.pad = 0;
    if (ok) lanes[line * P + lane] = li;
}

// Chunk transfer matrices (zero-input maps across one lane's chunk), FP64
// products stored as FP32: forward causal A_{b-1}..A_a, forward anticausal
// A_a..A_{b-1} (zero if the chunk holds a segment end), adjoint causal
// (A_a..A_{b-1})^T, adjoint anticausal (A_{b-1}..A_a)^T (zero if a segment
// end).  Empty chunks get identities.
__global__ void xfer_kernel(int64_t nrec, int64_t n, int64_t C, int P, int order,
                            const float4 *__restrict__ coef, float *__restrict__ xfer)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nrec) return;
    const int64_t line = idx / P, lane = idx - line * P;
    const int64_t a = lane * C, b = min(a + C, n);
    const float4 *cf = coef + line * n;
    const int M = order == 3 ? 9 : 1;
    double F[9], Pa[9], A[9], T[9];
    for (int k = 0; k < M; ++k) F[k] = Pa[k] = (order == 3) ? ((k % 4 == 0) ? 1.0 : 0.0) : 1.0;
    bool re = false;
    for (int64_t k = a; k < b; ++k) {
        step_matrix(cf[k], A, order);
        re = re || (__float_as_uint(cf[k].x) >> 31);
        if (order == 3) {
            mm3(A, F, T);
            for (int q = 0; q < 9; ++q) F[q] = T[q];
            mm3(Pa, A, T);
            for (int q = 0; q < 9; ++q) Pa[q] = T[q];
        } else {
            F[0] *= A[0];
            Pa[0] *= A[0];
        }
    }
    float *o = xfer + idx * (4 * M);
    for (int k = 0; k < M; ++k) {
        const int tr = order == 3 ? (k % 3) * 3 + k / 3 : 0;   // transpose index
        o[k] = (float)F[k];
        o[M + k] = re ? 0.f : (float)Pa[k];
        o[2 * M + k] = (float)Pa[tr];
        o[3 * M + k] = re ? 0.f : (float)F[tr];
    }
}

// Tables of the register-resident kernel for chunks of C points, P lanes per
// line (rf_reg.cuh), from the line-major coefficients: the interleaved
// coefficients with land (and points past the line's end) (0, 0, 0, -1), each
// lane's segment-end, segment-start and land bits with the rank of its first
// segment end on the line, and the four chunk transfer matrices in FP64
// products stored as FP32.  A transfer is zero if the chunk holds land (the
// reset factor clears the state there) or a segment end (the recorded state
// leaves the line there, and the anticausal start state replaces whatever
// arrives), and an anticausal-direction one also if it holds a segment
// start.  Otherwise, with A_k = J - 1 (e, c1, c2)_k the one-step
// matrix of point k: forward causal A_{b-1}..A_a, forward anticausal
// A_a..A_{b-1}, adjoint causal (A_a..A_{b-1})^T, adjoint anticausal
// (A_{b-1}..A_a)^T.  P threads per line; the P threads of a line lie in one
// warp (P divides 32), and a warp's lines past the end work on the last line
// and write nothing.
__global__ void reg_tables_kernel(int64_t nlines, int64_t n, int C, int P, int order,
                                  const float4 *__restrict__ coef, float4 *__restrict__ rc,
                                  RegLane *__restrict__ lanes, float *__restrict__ xfer)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t warp_line0 = (t & ~(int64_t)31) / P;
    if (warp_line0 >= nlines) return;   // whole warps past the end exit together
    const int64_t line0 = t / P;
    const int lane = (int)(t % P);
    const bool ok = line0 < nlines;
    const int64_t line = ok ? line0 : nlines - 1;
    const float4 *src = coef + line * n;
    const int64_t a = (int64_t)lane * C;
    u64 ends = 0, starts = 0, land = 0;
    double F[9], Pa[9];
    for (int k = 0; k < 9; ++k) F[k] = Pa[k] = (k % 4 == 0) ? 1.0 : 0.0;
    for (int k = 0; k < C; ++k) {
        const int64_t pos = a + k;
        float4 c = pos < n ? src[pos] : make_float4(0.f, 0.f, 0.f, -1.f);
        const bool sea = c.x != 0.f;
        if (sea && (__float_as_uint(c.x) >> 31)) ends |= 1ull << k;
        if (sea && (pos == 0 || src[pos - 1].x == 0.f)) starts |= 1ull << k;
        if (sea) {
            c.x = fabsf(c.x);
        } else {
            land |= 1ull << k;
            c = make_float4(0.f, 0.f, 0.f, -1.f);   // with g = 0: maps any state to zero
        }
        if (ok) rc[(line * C + k) * P + lane] = c;
        const double e = -(double)c.y, c1 = -(double)c.z, c2 = -(double)c.w;
        double A[9], T[9];
        if (order == 3) {
            const double J[9] = {1, 1, 1, 0, 1, 1, 0, 0, 1};
            const double kv[3] = {e, c1, c2};
            for (int r = 0; r < 3; ++r)
                for (int q = 0; q < 3; ++q) A[3 * r + q] = J[3 * r + q] - kv[q];
            mm3(A, F, T);
            for (int q = 0; q < 9; ++q) F[q] = T[q];
            mm3(Pa, A, T);
            for (int q = 0; q < 9; ++q) Pa[q] = T[q];
        } else {
            F[0] *= 1.0 - e;
            Pa[0] *= 1.0 - e;
        }
    }
    const bool zc = land != 0 || ends != 0, za = zc || starts != 0;
    const int M = order == 3 ? 9 : 1;
    if (ok) {
        float *o = xfer + (line * P + lane) * (4 * M);
        for (int k = 0; k < M; ++k) {
            const int tr = order == 3 ? (k % 3) * 3 + k / 3 : 0;   // transpose index
            o[k] = zc ? 0.f : (float)F[k];
            o[M + k] = za ? 0.f : (float)Pa[k];
            o[2 * M + k] = zc ? 0.f : (float)Pa[tr];
            o[3 * M + k] = za ? 0.f : (float)F[tr];
        }
    }
    const int nre = __popcll((long long)ends);
    int incl = nre;
    for (int d = 1; d < P; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, d, P);
        if (lane >= d) incl += v;
    }
    if (ok) {
        RegLane li;
        li.ends = ends;
        li.starts = starts;
        li.land = land;
        li.rank0 = incl - nre;
        li.nre = nre;
        lanes[line * P + lane] = li;
    }
}

// Imaginary points at a coast: ceil(img_factor sigma); -1 marks the
// infinite imaginary sea (img_factor = +inf), whose map is the closed-form
// limit.
int n_imaginary(double img_factor, float sigma)
{
    if (!(img_factor > 0.0)) return 0;
    if (std::isinf(img_factor)) return -1;
    return (int)std::ceil(img_factor * (double)sigma);
}

// Host analysis of one domain: validate length scales at sea points, then
// for each direction number the segments (runs of sea points) consecutively
// along each line, line after line, level after level, with the length
// scales and imaginary points at both ends.  base[d][lev*nlines + line] is
// the index of a line's first segment (base has one extra final entry: the
// total).
rf_status analyse(const rf_grid &g, int64_t ncl, const std::vector<uint8_t> &mask,
                  const std::vector<float> &Lx, const std::vector<float> &Ly,
                  double img_factor, std::vector<int32_t> base[2],
                  std::vector<TailSpec> sp[2], int max_re[2], int max_ends[2])
{
    const int64_t nx = g.nx, ny = g.ny, plane = nx * ny;
    base[0].assign((size_t)(ncl * ny + 1), 0);
    base[1].assign((size_t)(ncl * nx + 1), 0);
    max_re[0] = max_re[1] = 0;
    max_ends[0] = max_ends[1] = 0;
    // segment ends per line, with or without imaginary points (the register
    // kernel's record slots)
    for (int64_t k = 0; k < ncl; ++k) {
        const uint8_t *m = mask.data() + (g.mask_nz > 1 ? k : 0) * plane;
        for (int64_t j = 0; j < ny; ++j) {
            int cnt = 0;
            for (int64_t i = 0; i < nx; ++i)
                cnt += m[j * nx + i] && (i == nx - 1 || !m[j * nx + i + 1]);
            max_ends[0] = std::max(max_ends[0], cnt);
        }
        for (int64_t i = 0; i < nx; ++i) {
            int cnt = 0;
            for (int64_t j = 0; j < ny; ++j)
                cnt += m[j * nx + i] && (j == ny - 1 || !m[(j + 1) * nx + i]);
            max_ends[1] = std::max(max_ends[1], cnt);
        }
    }
    for (int64_t k = 0; k < ncl; ++k) {
        const uint8_t *m = mask.data() + (g.mask_nz > 1 ? k : 0) * plane;
        const float *lx = Lx.data() + (g.L_nz > 1 ? k : 0) * plane;
        const float *ly = Ly.data() + (g.L_nz > 1 ? k : 0) * plane;
        for (int64_t p = 0; p < plane; ++p) {
            if (!m[p]) continue;
            if (!(lx[p] > 0.f) || !std::isfinite(lx[p])) return RF_EINVAL;
            if (!(ly[p] > 0.f) || !std::isfinite(ly[p])) return RF_EINVAL;
        }
        const bool maps = img_factor > 0.0;
        for (int64_t j = 0; j < ny; ++j) {          // x lines: rows
            base[0][(size_t)(k * ny + j)] = (int32_t)sp[0].size();
            int cnt = 0;
            float sh = 0.f;
            for (int64_t i = 0; i < nx && maps; ++i) {
                const int64_t p = j * nx + i;
                if (m[p] && (i == 0 || !m[p - 1])) sh = lx[p];
                if (m[p] && (i == nx - 1 || !m[p + 1])) {
                    sp[0].push_back({lx[p], n_imaginary(img_factor, lx[p]), sh,
                                     n_imaginary(img_factor, sh)});
                    ++cnt;
                }
            }
            max_re[0] = std::max(max_re[0], cnt);
            if (sp[0].size() >= (size_t)INT32_MAX) return RF_EINVAL;
        }
        for (int64_t i = 0; i < nx; ++i) {          // y lines: columns
            base[1][(size_t)(k * nx + i)] = (int32_t)sp[1].size();
            int cnt = 0;
            float sh = 0.f;
            for (int64_t j = 0; j < ny && maps; ++j) {
                const int64_t p = j * nx + i;
                if (m[p] && (j == 0 || !m[p - nx])) sh = ly[p];
                if (m[p] && (j == ny - 1 || !m[p + nx])) {
                    sp[1].push_back({ly[p], n_imaginary(img_factor, ly[p]), sh,
                                     n_imaginary(img_factor, sh)});
                    ++cnt;
                }
            }
            max_re[1] = std::max(max_re[1], cnt);
            if (sp[1].size() >= (size_t)INT32_MAX) return RF_EINVAL;
        }
    }
    base[0].back() = (int32_t)sp[0].size();
    base[1].back() = (int32_t)sp[1].size();
    return RF_OK;
}

int64_t smem_stride(int64_t n)
{
    return n + ((4 - n % 32) + 32) % 32;   // row stride = 4 (mod 32) floats
}

// Lanes per line and chunk length of the tile kernel for line length n.
// Third-order lines of at most kShortLine points take 16 lanes (two lines
// per warp): chunks of up to 33 points instead of half that, and a scan over
// 16 lanes (one step fewer, over twice the points).  On short lines the
// per-chunk work (two 3x3 scans, the re-runs' start, the segment-end
// records) dominates a 32-lane chunk; from about 500 points on, the halved
// parallelism of 16 lanes costs more than it saves.  The first-order filter
// keeps 32 lanes: its scans are cheap.  C is odd, so the lanes' shared-memory
// accesses fall in distinct banks.  R = 0 marks lines too long for the tile
// kernel.
constexpr int64_t kShortLine = 512;

void choose_chunk(Dir &q, int order)
{
    q.P = order == 3 && q.n <= kShortLine ? 16 : 32;
    q.C = (q.n + q.P - 1) / q.P;
    if (q.C % 2 == 0) ++q.C;
    q.R = q.C <= kMaxChunk ? 1 : 0;   // R > 0 marks "tile kernel usable"
}

// (lines per CTA, slices per thread, lanes per line) shapes the tile kernel
// is built for (rf_launch_impl.cuh), in order of preference; a direction
// uses the shapes with its own lanes per line.
constexpr TileShape kShapesY[] = {
    {8, 4, 32},  {8, 2, 32},  {4, 4, 32},  {8, 1, 32},  {2, 4, 32},  {1, 4, 32},
    {1, 1, 32},  {1, 8, 32},  {2, 8, 32},  {4, 8, 32},  {8, 8, 32},  {16, 4, 32},
    {16, 8, 32}, {16, 4, 16}, {8, 4, 16},  {16, 8, 16}, {8, 8, 16},  {4, 4, 16},
    {16, 2, 16}, {8, 2, 16},  {8, 1, 16}};
constexpr TileShape kShapesX[] = {
    {4, 4, 32},  {8, 4, 32},  {2, 4, 32},  {8, 2, 32},  {8, 1, 32},  {1, 4, 32},
    {1, 1, 32},  {1, 8, 32},  {2, 8, 32},  {4, 8, 32},  {8, 8, 32},  {16, 4, 32},
    {16, 8, 32}, {4, 4, 16},  {8, 4, 16},  {16, 4, 16}, {8, 8, 16},  {16, 8, 16},
    {8, 2, 16},  {16, 2, 16}, {8, 1, 16}};

// Chunking of the register-resident kernel for one direction: the first
// built shape (kRegShapes) with P C >= n.  None (P = 0) for per-level
// coefficients, constant-extension coasts, longer lines, segment-end
// records that do not fit shared memory, and the third-order y pass (whose
// column strips the tile kernel filters faster: measured on the regional
// and the ragged batches).  The choice depends on the line and the options
// alone, never on tuning or batching.
RegShape reg_shape_for(const rf_plan_ *p, const Domain &D, const Dir &q, int dir)
{
    if (D.ncl != 1 || plan_cst(p) || q.n > 1024) return RegShape{0, 0};
    if (p->opt.order == 3 && dir == 1) return RegShape{0, 0};
    RegShape best{0, 0};
    for (const RegShape &s : kRegShapes)
        if ((int64_t)s.C * s.P >= q.n) {
            best = s;
            break;
        }
    if (best.P == 0) return best;
    if (reg_smem_bytes(dir, p->opt.order, best.C, best.P, kRegWarps, q.max_ends, reg_pairs(p->opt.order),
                       plan_carry(p) ? 2 + 2 * p->opt.iters : 0) > (int64_t)kSmemMax)
        return RegShape{0, 0};
    return best;
}

// Row-major copy of a direction's line-major coefficients, [n][nlines]
// (for the streaming column kernel).
__global__ void transpose_coef_kernel(int64_t nlines, int64_t n, const float4 *__restrict__ coef,
                                      float4 *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nlines * n) return;
    const int64_t r = i / nlines, line = i % nlines;
    out[i] = coef[line * n + r];
}

// The streaming column kernel serves the third-order y pass of 2-D
// coefficients with zero-input coasts whose columns have few enough
// segment ends for its per-thread records, on domains with at least
// kStreamMinWork columns x levels: below that its whole-column threads are
// too few to hide their serial chain of 2 ny steps, and the chunked tile
// kernel is faster (a 256 x 128 single-level impulse: 25.5 against 39.6 us
// per application).  A fixed rule per domain, so a domain's results do not
// depend on the batch it is in.
constexpr int64_t kStreamMinWork = 16384;

bool stream_ok(const rf_plan_ *p, const Domain &D, const Dir &q, int dir)
{
    return p->opt.order == 3 && dir == 1 && D.ncl == 1 && !plan_cst(p) &&
           q.max_ends <= kStreamMaxEnds && D.g.nx * D.g.nz >= kStreamMinWork;
}

rf_status build_dir(rf_plan_ *P, Domain &D, int dir, const uint8_t *mask_dev,
                    const float *L_dev, const std::vector<int32_t> &base,
                    const std::vector<TailSpec> &sp, int max_re, cudaStream_t st)
{
    const rf_grid &g = D.g;
    Dir &q = D.d[dir];
    q.dir = dir;
    q.n = dir == 0 ? g.nx : g.ny;
    q.nlines = dir == 0 ? g.ny : g.nx;
    q.pt_stride = dir == 0 ? 1 : g.nx;
    q.line_stride = dir == 0 ? g.nx : 1;
    q.ntail = (int64_t)sp.size();
    q.max_re = max_re;
    q.cst = (P->opt.flags & RF_FLAG_COAST_CONSTANT) && P->opt.img_factor > 0.0;
    choose_chunk(q, P->opt.order);
    const int64_t plane = g.nx * g.ny, ncl = D.ncl;
    const int o = P->opt.order, K = P->opt.iters, nm = P->opt.norm;
    const int qc = (P->opt.flags & RF_FLAG_Q_CORRECTED) ? 1 : 0;
    const int XS = o == 3 ? 36 : 4;

    RF_TRY(dev_alloc(&q.coef, ncl * plane, &P->bytes));
    RF_TRY(dev_alloc(&q.tail_base, (int64_t)base.size(), &P->bytes));
    RF_TRY(dev_alloc(&q.tmap, 9 * q.ntail, &P->bytes));
    if (q.cst) RF_TRY(dev_alloc(&q.cvec, 2 * q.ntail, &P->bytes));
    if (q.R > 0) {
        RF_TRY(dev_alloc(&q.xfer, ncl * q.nlines * q.P * XS, &P->bytes));
        RF_TRY(dev_alloc(&q.coef_il_base, ncl * q.nlines * q.C * q.P + 2 * kCoefGuard, &P->bytes));
        RF_TRY(dev_alloc(&q.lanes, ncl * q.nlines * q.P, &P->bytes));
        q.coef_il = q.coef_il_base + kCoefGuard;
        RF_TRY(cuda_status(cudaMemsetAsync(q.coef_il_base, 0,
                                           sizeof(float4) * (size_t)(ncl * q.nlines * q.C * q.P +
                                                                     2 * kCoefGuard), st)));
    }
    RF_TRY(cuda_status(cudaMemcpyAsync(q.tail_base, base.data(), base.size() * 4,
                                       cudaMemcpyHostToDevice, st)));
    const int64_t npts = ncl * plane;
    coef_lines_kernel<<<(unsigned)((npts + 255) / 256), 256, 0, st>>>(
        ncl, g.nx, g.ny, dir, mask_dev, g.mask_nz, L_dev, g.L_nz, o, K, nm, qc, q.coef);
    RF_TRY(cuda_status(cudaGetLastError()));
    if (q.R > 0) {
        const int64_t nrec = ncl * q.nlines * q.P;
        xfer_kernel<<<(unsigned)((nrec + 127) / 128), 128, 0, st>>>(nrec, q.n, q.C, q.P, o,
                                                                      q.coef, q.xfer);
        RF_TRY(cuda_status(cudaGetLastError()));
        const int64_t nl = ncl * q.nlines, lpb = 128 / q.P;
        interleave_kernel<<<(unsigned)((nl + lpb - 1) / lpb), 128, 0, st>>>(
            nl, q.n, (int)q.C, q.P, q.coef, q.coef_il, q.lanes);
        RF_TRY(cuda_status(cudaGetLastError()));
    }
    q.rsh = reg_shape_for(P, D, q, dir);
    if (stream_ok(P, D, q, dir)) {
        RF_TRY(dev_alloc(&q.tcoef, q.nlines * q.n, &P->bytes));
        transpose_coef_kernel<<<(unsigned)((q.nlines * q.n + 255) / 256), 256, 0, st>>>(
            q.nlines, q.n, q.coef, q.tcoef);
        RF_TRY(cuda_status(cudaGetLastError()));
    }
    if (q.rsh.P > 0) {
        const int64_t nrec = q.nlines * q.rsh.P;
        RF_TRY(dev_alloc(&q.rcoef, nrec * q.rsh.C, &P->bytes));
        RF_TRY(dev_alloc(&q.rlanes, nrec, &P->bytes));
        RF_TRY(dev_alloc(&q.rxfer, nrec * 4 * (o == 3 ? 9 : 1), &P->bytes));
        reg_tables_kernel<<<(unsigned)((nrec + 127) / 128), 128, 0, st>>>(
            q.nlines, q.n, q.rsh.C, q.rsh.P, o, q.coef, q.rcoef, q.rlanes, q.rxfer);
        RF_TRY(cuda_status(cudaGetLastError()));
    }
    if (!sp.empty()) {
        TailSpec *dsp = nullptr;
        int64_t dummy = 0;
        RF_TRY(dev_alloc(&dsp, (int64_t)sp.size(), &dummy));
        rf_status s = cuda_status(cudaMemcpyAsync(dsp, sp.data(), sp.size() * sizeof(TailSpec),
                                                  cudaMemcpyHostToDevice, st));
        if (s == RF_OK) {
            tail_kernel<<<(unsigned)((q.ntail + 127) / 128), 128, 0, st>>>(q.ntail, dsp, q.tmap,
                                                                           q.cvec, o, K, nm, qc);
            s = cuda_status(cudaGetLastError());
        }
        if (s == RF_OK) s = cuda_status(cudaStreamSynchronize(st));
        cudaFree(dsp);
        RF_TRY(s);
    }
    if (plan_carry(P) && q.ntail > 0) {
        // history weights of the carried coasts, FP64 on the host (the
        // infinite imaginary sea is cut where the oracle cuts it)
        q.kc = K;
        const int km = K - 1;
        std::vector<float> hw((size_t)(4 * q.ntail * km));
        std::vector<double> buf, w((size_t)km);
        for (int adj = 0; adj < 2; ++adj)
            for (int64_t i = 0; i < q.ntail; ++i)
                for (int side = 0; side < 2; ++side) {   // 0: the end (mu), 1: the start (lambda)
                    const double sg = side == 0 ? sp[(size_t)i].sigma : sp[(size_t)i].sigma_h;
                    const int ni = side == 0 ? sp[(size_t)i].n_img : sp[(size_t)i].n_h;
                    const int64_t n = ni < 0 ? (int64_t)std::ceil(60.0 * (1.0 + 2.0 * sg)) : ni;
                    buf.resize((size_t)(2 * n + 2));
                    carry_weights_fp64(sg, n, K, nm, adj != 0, side == 0, buf.data(), w.data());
                    for (int d = 0; d < km; ++d)
                        hw[(((size_t)adj * q.ntail + i) * 2 + side) * km + d] = (float)w[(size_t)d];
                }
        RF_TRY(dev_alloc(&q.carry, (int64_t)hw.size(), &P->bytes));
        RF_TRY(cuda_status(cudaMemcpyAsync(q.carry, hw.data(), hw.size() * sizeof(float),
                                           cudaMemcpyHostToDevice, st)));
        RF_TRY(cuda_status(cudaStreamSynchronize(st)));   // hw is released below
    }
    return RF_OK;
}

rf_status build_domain(rf_plan_ *P, Domain &D, const uint8_t *mask_dev,
                       const float *Lx_dev, const float *Ly_dev, cudaStream_t st)
{
    const rf_grid &g = D.g;
    const int64_t plane = g.nx * g.ny;
    D.ncl = (g.mask_nz > 1 || g.L_nz > 1) ? g.nz : 1;
    std::vector<uint8_t> hm((size_t)(g.mask_nz * plane));
    std::vector<float> hx((size_t)(g.L_nz * plane)), hy((size_t)(g.L_nz * plane));
    RF_TRY(cuda_status(cudaMemcpyAsync(hm.data(), mask_dev, hm.size(),
                                       cudaMemcpyDeviceToHost, st)));
    RF_TRY(cuda_status(cudaMemcpyAsync(hx.data(), Lx_dev, hx.size() * 4,
                                       cudaMemcpyDeviceToHost, st)));
    RF_TRY(cuda_status(cudaMemcpyAsync(hy.data(), Ly_dev, hy.size() * 4,
                                       cudaMemcpyDeviceToHost, st)));
    RF_TRY(cuda_status(cudaStreamSynchronize(st)));
    for (auto &v : hm) v = v ? 1 : 0;
    std::vector<int32_t> base[2];
    std::vector<TailSpec> sp[2];
    int max_re[2], max_ends[2];
    RF_TRY(analyse(g, D.ncl, hm, hx, hy, P->opt.img_factor, base, sp, max_re, max_ends));
    D.d[0].max_ends = max_ends[0];
    D.d[1].max_ends = max_ends[1];
    RF_TRY(build_dir(P, D, 0, mask_dev, Lx_dev, base[0], sp[0], max_re[0], st));
    RF_TRY(build_dir(P, D, 1, mask_dev, Ly_dev, base[1], sp[1], max_re[1], st));
    return cuda_status(cudaStreamSynchronize(st));
}

rf_status ensure(float **buf, int64_t *have, int64_t need, int64_t *bytes)
{
    if (need <= *have) return RF_OK;
    cudaFree(*buf);
    *bytes -= *have * 4;
    *have = 0;
    RF_TRY(dev_alloc(buf, need, bytes));
    *have = need;
    return RF_OK;
}

// ------------------------------------------------------------------ apply
int num_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 1;
        }
    }
    return sms;
}

// Complete a launch configuration whose shape and buffer count are set:
// shared memory, resident CTAs per SM, and the CTA rows along the slices
// (about two waves of CTAs; one row per level when the coefficients differ
// per level).  False if the shape does not fit or the slices per CTA are
// fewer than B.
template <int ORDER, bool ADJ>
bool finish_cfg(const Domain &D, const Dir &q, int64_t nvar, int64_t nk, LaunchCfg &L)
{
    const int64_t nslices = nvar * nk;
    const int64_t per_cta = D.ncl > 1 ? nvar : nslices;
    if (q.R == 0 || L.sh.P != q.P || (L.sh.B > 1 && L.sh.B > per_cta)) return false;
    L.smem = (size_t)tile_smem_bytes(L.sh.R, L.sh.B, smem_stride(q.n), q.max_re, L.nbuf,
                                     rec_floats(q));
    if (L.smem > kSmemMax) return false;
    L.occ = shape_occupancy<ORDER, ADJ, false>(L.sh, q.cst, L.smem);
    if (L.occ < 1) return false;
    L.tile = true;
    if (D.ncl > 1) {
        L.groups = nk;
    } else {
        const int64_t gx = (q.nlines + L.sh.R - 1) / L.sh.R;
        const int64_t target = 2 * (int64_t)num_sms() * L.occ;
        int64_t groups = (target + gx - 1) / gx;
        groups = std::min<int64_t>(groups, (nslices + L.sh.B - 1) / L.sh.B);
        L.groups = std::max<int64_t>(1, std::min<int64_t>(groups, 65535));
    }
    return true;
}

// Configuration of the register-resident kernel for one pass of nvar
// variables and nk levels, if the direction has its tables and the grid fits.
template <int ORDER, bool ADJ>
bool reg_cfg(const Dir &q, int64_t nvar, int64_t nk, LaunchCfg &L)
{
    if (q.rsh.P == 0) return false;
    const int64_t ngroups = (nvar * nk + 2 * reg_pairs(ORDER) - 1) / (2 * reg_pairs(ORDER));
    if ((q.dir == 0 ? (ngroups + kRegWarps - 1) / kRegWarps : ngroups) > 65535) return false;
    L = LaunchCfg{};
    L.reg = true;
    const bool car = ORDER == 1 && q.kc > 0;
    L.smem = (size_t)reg_smem_bytes(q.dir, ORDER, q.rsh.C, q.rsh.P, kRegWarps, q.max_ends,
                                    reg_pairs(ORDER), car ? 2 + 2 * q.kc : 0);
    if (car)
        L.occ = q.dir == 0 ? reg_occupancy<1, ADJ, 0, true>(q.rsh, L.smem)
                           : reg_occupancy<1, ADJ, 1, true>(q.rsh, L.smem);
    else
        L.occ = q.dir == 0 ? reg_occupancy<ORDER, ADJ, 0>(q.rsh, L.smem)
                           : reg_occupancy<ORDER, ADJ, 1>(q.rsh, L.smem);
    return L.occ > 0;
}

// Arguments of the streaming column kernel for one pass of one domain.
StreamArgs stream_args(const Domain &D, const Dir &q, const float *in, float *out, int64_t nvar,
                       int64_t k0, int64_t nk)
{
    StreamArgs a{};
    a.in = in;
    a.out = out;
    a.coef = q.tcoef;
    a.tail_base = q.tail_base;
    a.tmap = q.ntail > 0 ? q.tmap : nullptr;
    a.n = q.n;
    a.ncols = q.nlines;
    a.plane = D.g.nx * D.g.ny;
    a.nz = D.g.nz;
    a.k0 = k0;
    a.nk = nk;
    a.nslices = nvar * nk;
    a.npairs = (a.nslices + 1) / 2;
    a.scratch = q.max_ends;
    return a;
}

// Configuration of the streaming column kernel, if the direction has it.
template <int ORDER>
bool stream_cfg(const Dir &q, LaunchCfg &L)
{
    if (ORDER != 3 || !q.tcoef) return false;
    L = LaunchCfg{};
    L.strm = true;
    L.occ = 1;
    return true;
}

// Default (untuned) configuration: the register-resident kernel where it
// applies; else the first tile shape in the direction's preference list
// whose single-buffered shared memory allows two CTAs per SM, else the
// first that fits at all; the long-line kernel if none does.
template <int ORDER, bool ADJ>
LaunchCfg launch_cfg(const Domain &D, const Dir &q, int64_t nvar, int64_t nk)
{
    {
        LaunchCfg L;
        if (reg_cfg<ORDER, ADJ>(q, nvar, nk, L)) return L;
        if (stream_cfg<ORDER>(q, L)) return L;
    }
    if (q.kc > 0) return LaunchCfg{};   // carried coasts: the long-line kernel
    const int64_t ss = smem_stride(q.n);
    for (int pass = 0; pass < 2; ++pass) {
        const size_t cap = pass == 0 ? kSmemTarget : kSmemMax;
        for (const TileShape &s : q.pt_stride != 1 ? kShapesY : kShapesX) {
            if ((size_t)tile_smem_bytes(s.R, s.B, ss, q.max_re, 1, rec_floats(q)) > cap) continue;
            LaunchCfg L;
            L.sh = s;
            L.nbuf = 1;
            if (finish_cfg<ORDER, ADJ>(D, q, nvar, nk, L)) return L;
        }
    }
    return LaunchCfg{};
}

// Every tile configuration (shape and buffer count) that fits, for tuning.
template <int ORDER, bool ADJ>
std::vector<LaunchCfg> launch_candidates(const Domain &D, const Dir &q, int64_t nvar,
                                         int64_t nk)
{
    std::vector<LaunchCfg> out;
    {
        // where the register kernel applies it is the only candidate: the
        // kernel (hence the arithmetic) depends on the line length and the
        // options alone, never on tuning
        LaunchCfg L;
        if (reg_cfg<ORDER, ADJ>(q, nvar, nk, L) || stream_cfg<ORDER>(q, L)) {
            out.push_back(L);
            return out;
        }
        if (q.kc > 0) {   // carried coasts: the long-line kernel only
            out.push_back(LaunchCfg{});
            return out;
        }
    }
    for (const TileShape &s : kShapesY)
        for (int nbuf = 1; nbuf <= 2; ++nbuf) {
            LaunchCfg L;
            L.sh = s;
            L.nbuf = nbuf;
            if (finish_cfg<ORDER, ADJ>(D, q, nvar, nk, L)) out.push_back(L);
        }
    return out;
}

LaunchCfg launch_cfg_for(const rf_plan_ *p, const Domain &D, const Dir &q, int64_t nvar,
                         int64_t nk, bool adjoint)
{
    if (p->opt.order == 3)
        return adjoint ? launch_cfg<3, true>(D, q, nvar, nk) : launch_cfg<3, false>(D, q, nvar, nk);
    return adjoint ? launch_cfg<1, true>(D, q, nvar, nk) : launch_cfg<1, false>(D, q, nvar, nk);
}

// Levels per launch.  x and y of a batch of levels run back to back, so a
// batch whose field fits in L2 keeps the intermediate (the x pass output,
// read by the y pass) on chip, at the price of smaller launches.  All levels
// in one batch unless the autotuner found a batch size that is faster.
int64_t batch_levels(const Domain &D, int64_t nvar)
{
    for (const auto &e : D.batch)
        if (e.first == nvar) return e.second;
    return D.g.nz;
}

// Batch sizes the autotuner tries: all levels, and batches of about 96, 48
// and 24 MB of field.
std::vector<int64_t> batch_candidates(const Domain &D, int64_t nvar)
{
    const int64_t per_level = std::max<int64_t>(1, nvar * D.g.nx * D.g.ny * 4);
    std::vector<int64_t> out{D.g.nz};
    for (int64_t mb : {96, 48, 24}) {
        const int64_t nk = std::max<int64_t>(1, std::min<int64_t>(D.g.nz, (mb << 20) / per_level));
        if (std::find(out.begin(), out.end(), nk) == out.end()) out.push_back(nk);
    }
    return out;
}

// Arguments of the tile kernel for direction q of domain D.
TileArgs tile_args(const Domain &D, const Dir &q, const float *in, float *out, int64_t nvar,
                   int64_t k0, int64_t nk, int iters, int nbuf)
{
    TileArgs a{};
    a.in = in;
    a.out = out;
    a.coef = q.coef_il;
    a.lanes = q.lanes;
    a.xfer = q.xfer;
    a.tail_base = q.tail_base;
    a.tmap = q.tmap;
    a.cvec = q.cst ? q.cvec : nullptr;
    a.n = q.n;
    a.nlines = q.nlines;
    a.C = (int)q.C;
    a.pt_stride = q.pt_stride;
    a.line_stride = q.line_stride;
    a.plane = D.g.nx * D.g.ny;
    a.nz = D.g.nz;
    a.nvar = nvar;
    a.k0 = k0;
    a.nk = nk;
    a.ncl = D.ncl;
    a.iters = iters;
    a.smem_stride = (int)smem_stride(q.n);
    a.max_re = q.ntail > 0 ? q.max_re : 0;
    // x pass: rows start 16-byte aligned; y pass: rows of the grid do (so
    // groups of 4 adjacent columns can move as one 16-byte access)
    const bool al = ((uintptr_t)in % 16) == 0 && ((uintptr_t)out % 16) == 0;
    a.vec4 = al && (q.pt_stride == 1 ? q.n % 4 == 0 : q.pt_stride % 4 == 0);
    a.nbuf = nbuf;
    return a;
}

// Arguments of the register kernel for one pass of one domain.
template <int ORDER, bool ADJ>
RegArgs reg_args(const Domain &D, const Dir &q, const float *in, float *out, int64_t nvar,
                 int64_t k0, int64_t nk, int iters)
{
    const int64_t plane = D.g.nx * D.g.ny;
    RegArgs a{};
    a.in = in;
    a.out = out;
    a.coef = q.rcoef;
    a.lanes = q.rlanes;
    a.xfer = q.rxfer;
    a.tail_base = q.tail_base;
    a.tmap = q.ntail > 0 ? q.tmap : nullptr;
    a.n = q.n;
    a.nlines = q.nlines;
    a.nx = D.g.nx;
    a.plane = plane;
    a.nz = D.g.nz;
    a.k0 = k0;
    a.nk = nk;
    a.nslices = nvar * nk;
    a.ngroups = (a.nslices + 2 * reg_pairs(ORDER) - 1) / (2 * reg_pairs(ORDER));
    a.max_re = q.max_ends;
    a.vec4 = D.g.nx % 4 == 0 && ((uintptr_t)in % 16) == 0 && ((uintptr_t)out % 16) == 0;
    a.iters = iters;
    a.zero = 0;
    a.status = D.status;
    a.wait_polls = D.wait_polls ? *D.wait_polls : kRegWaitTries;
    const bool car = ORDER == 1 && q.kc > 0;
    a.kc = q.kc;
    a.rs = car ? 2 + 2 * q.kc : (ORDER == 3 ? 3 : 1);
    a.carry = car ? q.carry + (ADJ ? 2 * (q.kc - 1) * q.ntail : 0) : nullptr;
    return a;
}

template <int ORDER, bool ADJ>
void launch_dir(const Domain &D, const Dir &q, const LaunchCfg &L, const float *in,
                float *out, int64_t nvar, int64_t k0, int64_t nk, int iters, cudaStream_t st)
{
    const int64_t plane = D.g.nx * D.g.ny;
    if (L.reg) {
        const RegArgs a = reg_args<ORDER, ADJ>(D, q, in, out, nvar, k0, nk, iters);
        const bool car = ORDER == 1 && q.kc > 0;
        if (car) {
            if (q.dir == 0) reg_launch<1, ADJ, 0, true>(a, q.rsh, L.smem, st);
            else reg_launch<1, ADJ, 1, true>(a, q.rsh, L.smem, st);
        } else {
            if (q.dir == 0) reg_launch<ORDER, ADJ, 0>(a, q.rsh, L.smem, st);
            else reg_launch<ORDER, ADJ, 1>(a, q.rsh, L.smem, st);
        }
    } else if (L.strm) {
        stream_launch<ADJ>(stream_args(D, q, in, out, nvar, k0, nk), st);
    } else if (L.tile) {
        const TileArgs a = tile_args(D, q, in, out, nvar, k0, nk, iters, L.nbuf);
        launch_shape<ORDER, ADJ>(a, L.sh, q.cst, q.nlines, L.groups, L.smem, st);
    } else {
        LineArgs a{};
        a.in = in;
        a.out = out;
        a.coef = q.coef;
        a.tail_base = q.tail_base;
        a.tmap = q.tmap;
        a.cvec = q.cst ? q.cvec : nullptr;
        a.nr = rec_floats(q);
        a.tscr = D.tscr;
        a.kc = q.kc;
        a.carry = q.kc > 0 ? q.carry + (ADJ ? 2 * (q.kc - 1) * q.ntail : 0) : nullptr;
        a.n = q.n;
        a.nlines = q.nlines;
        a.pt_stride = q.pt_stride;
        a.line_stride = q.line_stride;
        a.plane = plane;
        a.nz = D.g.nz;
        a.nvar = nvar;
        a.k0 = k0;
        a.nk = nk;
        a.ntail = q.ntail;
        a.ncl = D.ncl;
        a.iters = iters;
        const int64_t threads = q.nlines * nvar * nk;
        line_kernel<ORDER, ADJ><<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(a);
    }
}

// True if a configuration runs the long-line kernel (which keeps its
// segment-end states in the domain's global scratch).
bool line_path(const LaunchCfg &L)
{
    return !L.tile && !L.reg && !L.strm;
}

// Launch configuration of direction dir for nvar variables and batches of
// nk levels: the tuned or cached one, else the default.
LaunchCfg cfg_of(const rf_plan_ *p, Domain &D, int dir, int64_t nvar, int64_t nk, bool adjoint)
{
    Dir &q = D.d[dir];
    for (const CfgEntry &e : q.cfgs)
        if (e.nvar == nvar && e.nk == nk && e.adjoint == adjoint) return e.cfg;
    const LaunchCfg c = launch_cfg_for(p, D, q, nvar, nk, adjoint);
    q.cfgs.push_back({nvar, nk, adjoint, c});
    return c;
}

// V_H (or its adjoint) on one domain, in batches of nkb levels.
// dry: choose the configurations and grow the scratch, but launch nothing
// (run before a stream capture, so the captured call allocates nothing).
rf_status apply_domain(rf_plan_ *p, Domain &D, const float *in, float *out, int nvar,
                       bool adjoint, int64_t nkb, bool dry, cudaStream_t st)
{
    const int64_t nz = D.g.nz;
    // global scratch for segment-end states, only for the long-line path
    int64_t nt = 0;
    for (int dir = 0; dir < 2; ++dir)
        if (line_path(cfg_of(p, D, dir, nvar, nkb, adjoint)) ||
            line_path(cfg_of(p, D, dir, nvar, nz - (nz - 1) / nkb * nkb, adjoint)))
            nt = std::max(nt, D.d[dir].ntail * (int64_t)rec_floats(D.d[dir]));
    rf_status s = ensure(&D.tscr, &D.tscr_floats, (int64_t)nvar * nz * nt, &p->bytes);
    if (s != RF_OK) return s;
    const int K = p->opt.iters;
    for (int64_t k0 = 0; k0 < nz; k0 += nkb) {
        if (dry) {
            cfg_of(p, D, 0, nvar, std::min(nkb, nz - k0), adjoint);
            cfg_of(p, D, 1, nvar, std::min(nkb, nz - k0), adjoint);
            continue;
        }
        const int64_t nk = std::min(nkb, nz - k0);
        for (int pass = 0; pass < 2; ++pass) {
            const int dir = adjoint ? 1 - pass : pass;   // forward x then y
            const float *src = pass == 0 ? in : out;
            const Dir &q = D.d[dir];
            const LaunchCfg L = cfg_of(p, D, dir, nvar, nk, adjoint);
            if (p->opt.order == 3) {
                if (adjoint) launch_dir<3, true>(D, q, L, src, out, nvar, k0, nk, 1, st);
                else launch_dir<3, false>(D, q, L, src, out, nvar, k0, nk, 1, st);
            } else {
                if (adjoint) launch_dir<1, true>(D, q, L, src, out, nvar, k0, nk, K, st);
                else launch_dir<1, false>(D, q, L, src, out, nvar, k0, nk, K, st);
            }
            s = cuda_status(cudaGetLastError());
            if (s != RF_OK) {
                if (p->sticky == RF_OK) p->sticky = s;
                return s;
            }
            ++p->launches;
        }
    }
    return RF_OK;
}

// ------------------------------------------------------ multi-domain launches
// The tile-kernel domains of one pass share a launch shape and the largest
// domain's shared memory.  A domain with fewer slices per CTA than B (the
// variables of one level when its coefficients differ per level) fills its
// groups partly, which costs idle slots but no correctness.
bool multi_fits(const rf_plan_ *p, int dir, int64_t nvar, TileShape sh, size_t *smem)
{
    (void)nvar;
    size_t m = 0;
    bool any = false;
    for (const Domain &D : p->dom) {
        const Dir &q = D.d[dir];
        if (q.R == 0 || q.P != sh.P || q.rsh.P > 0 || q.kc > 0 || q.tcoef) continue;   // launched on their own
        m = std::max(m, (size_t)tile_smem_bytes(sh.R, sh.B, smem_stride(q.n), q.max_re, 1,
                                                rec_floats(q)));
        any = true;
    }
    *smem = m;
    return any && m + 64 <= kSmemMax;   // the kernel's own static shared memory
}

template <int ORDER, bool ADJ>
bool multi_try(const rf_plan_ *p, int dir, int64_t nvar, TileShape sh, MultiCfg &c)
{
    size_t smem = 0;
    if (!multi_fits(p, dir, nvar, sh, &smem)) return false;
    const int occ = shape_occupancy<ORDER, ADJ, true>(sh, plan_cst(p), smem);
    if (occ < 1) return false;
    c = MultiCfg{nvar, ADJ, dir, sh.P, sh, smem, occ};
    return true;
}

bool multi_try_any(const rf_plan_ *p, int dir, int64_t nvar, bool adjoint, TileShape sh,
                   MultiCfg &c)
{
    if (p->opt.order == 3)
        return adjoint ? multi_try<3, true>(p, dir, nvar, sh, c)
                       : multi_try<3, false>(p, dir, nvar, sh, c);
    return adjoint ? multi_try<1, true>(p, dir, nvar, sh, c) : multi_try<1, false>(p, dir, nvar, sh, c);
}

// Shape of a pass over the domains with P lanes per line: tuned, cached, or
// the first of the direction's preference list that allows two CTAs and eight
// warps per SM with the largest domain's shared memory (else the first that
// fits).  occ = 0: no domain of the pass runs on the tile kernel with P.
MultiCfg multi_cfg(rf_plan_ *p, int dir, int64_t nvar, bool adjoint, int P)
{
    for (const MultiCfg &c : p->mcfg)
        if (c.nvar == nvar && c.adjoint == adjoint && c.dir == dir && c.P == P) return c;
    MultiCfg c{nvar, adjoint, dir, P, {0, 0, P}, 0, 0};
    bool found = false;
    for (int pass = 0; pass < 2 && !found; ++pass)
        for (const TileShape &sh : dir == 1 ? kShapesY : kShapesX) {
            MultiCfg t;
            if (sh.P == P && multi_try_any(p, dir, nvar, adjoint, sh, t) &&
                (pass == 1 || (t.smem <= kSmemTarget && t.occ * sh.R * sh.P / 32 >= 8))) {
                c = t;
                found = true;
                break;
            }
        }
    p->mcfg.push_back(c);
    return c;
}

// One pass (direction c.dir) over every tile-kernel domain with c.P lanes
// per line: persistent launches over work lists of at most kMaxMulti domains,
// the domains split evenly between the launches.
rf_status multi_pass(rf_plan_ *p, const MultiCfg &c, const float *const *src,
                     float *const *out, int nvar, bool adjoint, cudaStream_t st)
{
    std::vector<int> doms;
    for (size_t d = 0; d < p->dom.size(); ++d)
        if (p->dom[d].d[c.dir].R > 0 && p->dom[d].d[c.dir].P == c.P && p->dom[d].d[c.dir].rsh.P == 0 &&
            p->dom[d].d[c.dir].kc == 0 && !p->dom[d].d[c.dir].tcoef)
            doms.push_back((int)d);
    const int iters = p->opt.order == 3 ? 1 : p->opt.iters;
    const size_t nlaunch = (doms.size() + kMaxMulti - 1) / kMaxMulti;
    const size_t per = nlaunch ? (doms.size() + nlaunch - 1) / nlaunch : 0;
    for (size_t c0 = 0; c0 < doms.size(); c0 += per) {
        MultiArgs m{};
        m.ndom = (int)std::min(per, doms.size() - c0);
        m.queue = p->queue;
        int64_t total = 0;
        for (int k = 0; k < m.ndom; ++k) {
            const Domain &D = p->dom[doms[c0 + k]];
            const Dir &q = D.d[c.dir];
            const int d = doms[c0 + k];
            m.dom[k] = tile_args(D, q, src[d], out[d], nvar, 0, D.g.nz, iters, 1);
            m.gx[k] = (q.nlines + c.sh.R - 1) / c.sh.R;
            m.rows[k] = D.ncl > 1 ? D.g.nz : (nvar * D.g.nz + c.sh.B - 1) / c.sh.B;
            m.first[k] = total;
            total += m.gx[k] * m.rows[k];
        }
        m.first[m.ndom] = total;
        const unsigned grid = (unsigned)std::min<int64_t>(total, (int64_t)num_sms() * c.occ);
        RF_TRY(cuda_status(cudaMemsetAsync(p->queue, 0, sizeof(unsigned long long), st)));
        if (p->opt.order == 3) {
            if (adjoint) launch_multi<3, true>(m, c.sh, plan_cst(p), grid, c.smem, st);
            else launch_multi<3, false>(m, c.sh, plan_cst(p), grid, c.smem, st);
        } else {
            if (adjoint) launch_multi<1, true>(m, c.sh, plan_cst(p), grid, c.smem, st);
            else launch_multi<1, false>(m, c.sh, plan_cst(p), grid, c.smem, st);
        }
        const rf_status s = cuda_status(cudaGetLastError());
        if (s != RF_OK) {
            if (p->sticky == RF_OK) p->sticky = s;
            return s;
        }
        ++p->launches;
    }
    return RF_OK;
}

// One pass of the register-kernel domains of a batch: one launch per chunk
// shape (C, P) over all domains of that shape (in groups of kRegMulti), the
// CTAs of every domain's grid concatenated.
template <int ORDER, bool ADJ>
rf_status reg_multi_group(rf_plan_ *p, int dir, const std::vector<size_t> &ds,
                          const float *const *src, float *const *out, int nvar, cudaStream_t st)
{
    RegMulti m{};
    const RegShape sh = p->dom[ds[0]].d[dir].rsh;
    const bool car = ORDER == 1 && p->dom[ds[0]].d[dir].kc > 0;
    size_t smem = 0;
    m.nd = (int)ds.size();
    m.cta0[0] = 0;
    for (int i = 0; i < m.nd; ++i) {
        const Domain &D = p->dom[ds[(size_t)i]];
        const Dir &q = D.d[dir];
        m.dom[i] = reg_args<ORDER, ADJ>(D, q, src[ds[(size_t)i]], out[ds[(size_t)i]], nvar, 0,
                                        D.g.nz, ORDER == 3 ? 1 : p->opt.iters);
        const dim3 g = reg_grid(dir, sh, m.dom[i].nlines, m.dom[i].ngroups);
        m.gx[i] = (int)g.x;
        m.cta0[i + 1] = m.cta0[i] + (int64_t)g.x * g.y;
        smem = std::max(smem, (size_t)reg_smem_bytes(dir, ORDER, sh.C, sh.P, kRegWarps, q.max_ends,
                                                     reg_pairs(ORDER), car ? 2 + 2 * q.kc : 0));
    }
    if (m.cta0[m.nd] > INT32_MAX) return RF_EINVAL;
    const unsigned grid = (unsigned)m.cta0[m.nd];
    if (car) {
        if (dir == 0) reg_launch_multi<1, ADJ, 0, true>(m, sh, smem, grid, st);
        else reg_launch_multi<1, ADJ, 1, true>(m, sh, smem, grid, st);
    } else {
        if (dir == 0) reg_launch_multi<ORDER, ADJ, 0>(m, sh, smem, grid, st);
        else reg_launch_multi<ORDER, ADJ, 1>(m, sh, smem, grid, st);
    }
    const rf_status s = cuda_status(cudaGetLastError());
    if (s != RF_OK) {
        if (p->sticky == RF_OK) p->sticky = s;
        return s;
    }
    ++p->launches;
    return RF_OK;
}

rf_status reg_multi_pass(rf_plan_ *p, int dir, const float *const *src, float *const *out,
                         int nvar, bool adjoint, cudaStream_t st)
{
    // domains grouped by chunk shape, in plan order
    std::vector<std::pair<std::pair<int, int>, std::vector<size_t>>> groups;
    for (size_t d = 0; d < p->dom.size(); ++d) {
        const RegShape sh = p->dom[d].d[dir].rsh;
        if (sh.P == 0) continue;
        auto it = std::find_if(groups.begin(), groups.end(),
                               [&](const auto &g) { return g.first == std::make_pair(sh.C, sh.P); });
        if (it == groups.end()) {
            groups.push_back({{sh.C, sh.P}, {}});
            it = groups.end() - 1;
        }
        it->second.push_back(d);
    }
    for (const auto &g : groups)
        for (size_t i0 = 0; i0 < g.second.size(); i0 += kRegMulti) {
            const std::vector<size_t> ds(g.second.begin() + (ptrdiff_t)i0,
                                         g.second.begin() +
                                             (ptrdiff_t)std::min(g.second.size(), i0 + kRegMulti));
            rf_status s;
            if (p->opt.order == 3)
                s = adjoint ? reg_multi_group<3, true>(p, dir, ds, src, out, nvar, st)
                            : reg_multi_group<3, false>(p, dir, ds, src, out, nvar, st);
            else
                s = adjoint ? reg_multi_group<1, true>(p, dir, ds, src, out, nvar, st)
                            : reg_multi_group<1, false>(p, dir, ds, src, out, nvar, st);
            RF_TRY(s);
        }
    return RF_OK;
}

// One pass of the streaming-kernel domains of a batch: one launch over up
// to kStreamMulti domains, the CTAs of every domain's grid concatenated.
rf_status stream_multi_pass(rf_plan_ *p, int dir, const float *const *src, float *const *out,
                            int nvar, bool adjoint, cudaStream_t st)
{
    std::vector<size_t> ds;
    for (size_t d = 0; d < p->dom.size(); ++d)
        if (p->dom[d].d[dir].tcoef) ds.push_back(d);
    for (size_t i0 = 0; i0 < ds.size(); i0 += kStreamMulti) {
        StreamMulti m{};
        m.nd = (int)std::min<size_t>(kStreamMulti, ds.size() - i0);
        m.cta0[0] = 0;
        for (int i = 0; i < m.nd; ++i) {
            const Domain &D = p->dom[ds[i0 + (size_t)i]];
            m.dom[i] = stream_args(D, D.d[dir], src[ds[i0 + (size_t)i]], out[ds[i0 + (size_t)i]], nvar, 0,
                                   D.g.nz);
            const dim3 g = stream_grid(m.dom[i].ncols, m.dom[i].npairs);
            m.gx[i] = (int)g.x;
            m.cta0[i + 1] = m.cta0[i] + (int64_t)g.x * g.y;
        }
        if (m.cta0[m.nd] > INT32_MAX) return RF_EINVAL;
        if (adjoint) stream_launch_multi<true>(m, (unsigned)m.cta0[m.nd], st);
        else stream_launch_multi<false>(m, (unsigned)m.cta0[m.nd], st);
        const rf_status s = cuda_status(cudaGetLastError());
        if (s != RF_OK) {
            if (p->sticky == RF_OK) p->sticky = s;
            return s;
        }
        ++p->launches;
    }
    return RF_OK;
}

// Multi-domain application: x over all domains, then y over all domains
// (adjoint: y then x); the domains too long for the tile kernel in a
// direction run on the long-line kernel in the same pass.
rf_status apply_multi(rf_plan_ *p, const float *const *in, float *const *out, int nvar,
                      bool adjoint, bool dry, cudaStream_t st)
{
    if (!p->queue) RF_TRY(dev_alloc(&p->queue, 1, &p->bytes));
    // per direction one multi-domain configuration for each lanes-per-line
    // value (32 and, for the 3rd-RF, 16)
    const int nP = p->opt.order == 3 ? 2 : 1;
    MultiCfg cs[2][2];
    for (int dir = 0; dir < 2; ++dir)
        for (int k = 0; k < nP; ++k) cs[dir][k] = multi_cfg(p, dir, nvar, adjoint, k ? 16 : 32);
    // domains no multi-domain launch covers (lines too long for the tile
    // kernel, or no shape fits) launch on their own
    auto covered = [&](const Dir &q, int dir) {
        if (q.rsh.P > 0 || q.tcoef) return true;   // the multi-domain register / streaming launches below
        if (q.R == 0 || q.kc > 0 || q.tcoef) return false;   // long-line, carried-coast and streaming domains launch on their own
        for (int k = 0; k < nP; ++k)
            if (cs[dir][k].occ > 0 && cs[dir][k].P == q.P) return true;
        return false;
    };
    for (Domain &D : p->dom) {
        int64_t nt = 0;
        for (int dir = 0; dir < 2; ++dir) {
            const Dir &q = D.d[dir];
            if (covered(q, dir)) continue;
            if (q.R == 0 || line_path(cfg_of(p, D, dir, nvar, D.g.nz, adjoint)))
                nt = std::max(nt, q.ntail * (int64_t)rec_floats(q));
        }
        RF_TRY(ensure(&D.tscr, &D.tscr_floats, (int64_t)nvar * D.g.nz * nt, &p->bytes));
    }
    if (dry) return RF_OK;
    const int K = p->opt.iters;
    for (int pass = 0; pass < 2; ++pass) {
        const int dir = adjoint ? 1 - pass : pass;
        const float *const *src = pass == 0 ? in : (const float *const *)out;
        for (int k = 0; k < nP; ++k)
            if (cs[dir][k].occ > 0) RF_TRY(multi_pass(p, cs[dir][k], src, out, nvar, adjoint, st));
        RF_TRY(reg_multi_pass(p, dir, src, out, nvar, adjoint, st));
        RF_TRY(stream_multi_pass(p, dir, src, out, nvar, adjoint, st));
        for (size_t d = 0; d < p->dom.size(); ++d) {
            Domain &D = p->dom[d];
            const Dir &q = D.d[dir];
            if (covered(q, dir)) continue;
            const LaunchCfg L = q.R > 0 ? cfg_of(p, D, dir, nvar, D.g.nz, adjoint) : LaunchCfg{};
            if (p->opt.order == 3) {
                if (adjoint) launch_dir<3, true>(D, q, L, src[d], out[d], nvar, 0, D.g.nz, 1, st);
                else launch_dir<3, false>(D, q, L, src[d], out[d], nvar, 0, D.g.nz, 1, st);
            } else {
                if (adjoint) launch_dir<1, true>(D, q, L, src[d], out[d], nvar, 0, D.g.nz, K, st);
                else launch_dir<1, false>(D, q, L, src[d], out[d], nvar, 0, D.g.nz, K, st);
            }
            const rf_status s = cuda_status(cudaGetLastError());
            if (s != RF_OK) {
                if (p->sticky == RF_OK) p->sticky = s;
                return s;
            }
            ++p->launches;
        }
    }
    return RF_OK;
}

// Several domains go through the multi-domain launches unless the
// autotuner found the per-domain launches faster.
bool use_multi(const rf_plan_ *p, int64_t nvar)
{
    if (p->dom.size() < 2) return false;
    for (const auto &e : p->multi_pref)
        if (e.first == nvar) return e.second;
    return true;
}

rf_status apply_impl(rf_plan p, const float *const *in, float *const *out, int nvar,
                     bool adjoint, cudaStream_t st, bool dry = false)
{
    if (!p || !in || !out || nvar < 1) return RF_EINVAL;
    for (size_t d = 0; d < p->dom.size(); ++d)
        if (!in[d] || !out[d]) return RF_EINVAL;
    if (use_multi(p, nvar)) return apply_multi(p, in, out, nvar, adjoint, dry, st);
    for (size_t d = 0; d < p->dom.size(); ++d) {
        Domain &D = p->dom[d];
        RF_TRY(apply_domain(p, D, in[d], out[d], nvar, adjoint, batch_levels(D, nvar), dry, st));
    }
    return RF_OK;
}

// One launch of direction q with configuration L, for tuning.
void launch_any(const rf_plan_ *p, const Domain &D, const Dir &q, const LaunchCfg &L,
                const float *in, float *out, int64_t nvar, int64_t nk, bool adjoint,
                cudaStream_t st)
{
    const int K = p->opt.iters;
    if (p->opt.order == 3) {
        if (adjoint) launch_dir<3, true>(D, q, L, in, out, nvar, 0, nk, 1, st);
        else launch_dir<3, false>(D, q, L, in, out, nvar, 0, nk, 1, st);
    } else {
        if (adjoint) launch_dir<1, true>(D, q, L, in, out, nvar, 0, nk, K, st);
        else launch_dir<1, false>(D, q, L, in, out, nvar, 0, nk, K, st);
    }
}

std::vector<LaunchCfg> candidates_for(const rf_plan_ *p, const Domain &D, const Dir &q,
                                      int64_t nvar, int64_t nk, bool adjoint)
{
    if (p->opt.order == 3)
        return adjoint ? launch_candidates<3, true>(D, q, nvar, nk)
                       : launch_candidates<3, false>(D, q, nvar, nk);
    return adjoint ? launch_candidates<1, true>(D, q, nvar, nk)
                   : launch_candidates<1, false>(D, q, nvar, nk);
}

// Autotuner.  For every batch size of batch_candidates: time every candidate
// launch configuration of every direction on scratch fields (zeros; the work
// does not depend on the values) and keep the fastest, then time whole
// forward + adjoint applications with those configurations.  The batch size
// of the fastest application is kept.
rf_status tune_shapes(rf_plan_ *p, Domain &D, int nvar, int64_t nk, float *buf, int64_t nf,
                      cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st)
{
    for (int adj = 0; adj < 2; ++adj) {
        for (int dir = 0; dir < 2; ++dir) {
            Dir &q = D.d[dir];
            const std::vector<LaunchCfg> cands = candidates_for(p, D, q, nvar, nk, adj != 0);
            if (cands.empty()) continue;
            float best_ms = 0.f;
            LaunchCfg best;
            for (const LaunchCfg &L : cands) {
                launch_any(p, D, q, L, buf, buf + nf, nvar, nk, adj != 0, st);   // warm-up
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3; ++r)
                    launch_any(p, D, q, L, buf, buf + nf, nvar, nk, adj != 0, st);
                cudaEventRecord(e1, st);
                RF_TRY(cuda_status(cudaEventSynchronize(e1)));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (best_ms == 0.f || ms < best_ms) {
                    best_ms = ms;
                    best = L;
                }
            }
            bool found = false;
            for (CfgEntry &e : q.cfgs)
                if (e.nvar == nvar && e.nk == nk && e.adjoint == (adj != 0)) {
                    e.cfg = best;
                    found = true;
                }
            if (!found) q.cfgs.push_back({nvar, nk, adj != 0, best});
        }
    }
    return RF_OK;
}

rf_status tune_domain(rf_plan_ *p, Domain &D, int nvar, float *buf, int64_t nf, cudaEvent_t e0,
                      cudaEvent_t e1, cudaStream_t st)
{
    RF_TRY(cuda_status(cudaMemsetAsync(buf, 0, sizeof(float) * 2 * (size_t)nf, st)));
    const int64_t nz = D.g.nz;
    float best_ms = 0.f;
    int64_t best_nkb = nz;
    for (int64_t nkb : batch_candidates(D, nvar)) {
        // a full batch and the remainder
        RF_TRY(tune_shapes(p, D, nvar, nkb, buf, nf, e0, e1, st));
        const int64_t rest = nz - (nz - 1) / nkb * nkb;
        if (rest != nkb) RF_TRY(tune_shapes(p, D, nvar, rest, buf, nf, e0, e1, st));
        for (int rep = 0; rep < 3; ++rep) {   // one warm-up, then two timed
            if (rep == 1) cudaEventRecord(e0, st);
            RF_TRY(apply_domain(p, D, buf, buf + nf, nvar, false, nkb, false, st));
            RF_TRY(apply_domain(p, D, buf + nf, buf, nvar, true, nkb, false, st));
        }
        cudaEventRecord(e1, st);
        RF_TRY(cuda_status(cudaEventSynchronize(e1)));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms == 0.f || ms < best_ms) {
            best_ms = ms;
            best_nkb = nkb;
        }
    }
    bool found = false;
    for (auto &e : D.batch)
        if (e.first == nvar) {
            e.second = best_nkb;
            found = true;
        }
    if (!found) D.batch.push_back({nvar, best_nkb});
    return RF_OK;
}

// Multi-domain tuning: time every shape that fits for each pass, then whole
// forward + adjoint applications with multi-domain against per-domain
// launches, and keep the faster.
rf_status tune_multi(rf_plan_ *p, int nvar, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st)
{
    const size_t nd = p->dom.size();
    std::vector<float *> bufs(nd, nullptr);
    std::vector<const float *> ins(nd);
    std::vector<float *> outs(nd);
    rf_status s = RF_OK;
    int64_t dummy = 0;
    for (size_t d = 0; d < nd && s == RF_OK; ++d) {
        const Domain &D = p->dom[d];
        const int64_t nf = (int64_t)nvar * D.g.nz * D.g.nx * D.g.ny;
        s = dev_alloc(&bufs[d], 2 * nf, &dummy);
        if (s == RF_OK)
            s = cuda_status(cudaMemsetAsync(bufs[d], 0, sizeof(float) * 2 * (size_t)nf, st));
        ins[d] = bufs[d];
        outs[d] = bufs[d] + nf;
    }
    if (s == RF_OK && !p->queue) s = dev_alloc(&p->queue, 1, &p->bytes);
    auto elapsed = [&](float *ms) -> rf_status {
        cudaEventRecord(e1, st);
        RF_TRY(cuda_status(cudaEventSynchronize(e1)));
        cudaEventElapsedTime(ms, e0, e1);
        return RF_OK;
    };
    const int nP = p->opt.order == 3 ? 2 : 1;
    for (int adj = 0; adj < 2 && s == RF_OK; ++adj)
        for (int dir = 0; dir < 2 && s == RF_OK; ++dir)
            for (int k = 0; k < nP && s == RF_OK; ++k) {
                const int P = k ? 16 : 32;
                float best_ms = 0.f;
                MultiCfg best{nvar, adj != 0, dir, P, {0, 0, P}, 0, 0};
                for (const TileShape &sh : kShapesY) {
                    MultiCfg c;
                    if (sh.P != P || !multi_try_any(p, dir, nvar, adj != 0, sh, c)) continue;
                    s = multi_pass(p, c, ins.data(), outs.data(), nvar, adj != 0, st);   // warm-up
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < 3 && s == RF_OK; ++r)
                        s = multi_pass(p, c, ins.data(), outs.data(), nvar, adj != 0, st);
                    float ms = 0.f;
                    if (s == RF_OK) s = elapsed(&ms);
                    if (s != RF_OK) break;
                    if (best_ms == 0.f || ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
                if (s != RF_OK || best.occ == 0) continue;
                bool found = false;
                for (MultiCfg &e : p->mcfg)
                    if (e.nvar == nvar && e.adjoint == (adj != 0) && e.dir == dir && e.P == P) {
                        e = best;
                        found = true;
                    }
                if (!found) p->mcfg.push_back(best);
            }
    // multi-domain against per-domain launches
    float t[2] = {0.f, 0.f};
    for (int multi = 0; multi < 2 && s == RF_OK; ++multi) {
        p->multi_pref.erase(std::remove_if(p->multi_pref.begin(), p->multi_pref.end(),
                                           [&](const std::pair<int64_t, bool> &e) {
                                               return e.first == nvar;
                                           }),
                            p->multi_pref.end());
        p->multi_pref.push_back({nvar, multi != 0});
        for (int rep = 0; rep < 3 && s == RF_OK; ++rep) {   // one warm-up, then two timed
            if (rep == 1) cudaEventRecord(e0, st);
            s = apply_impl(p, ins.data(), outs.data(), nvar, false, st);
            if (s == RF_OK) s = apply_impl(p, (const float *const *)outs.data(), (float *const *)ins.data(), nvar, true, st);
        }
        if (s == RF_OK) s = elapsed(&t[multi]);
    }
    if (s == RF_OK) p->multi_pref.back().second = t[1] <= t[0];
    cudaStreamSynchronize(st);
    for (float *b : bufs) cudaFree(b);
    return s;
}

// ------------------------------------------------------ host-buffer apply
// Copy streams and events of the host-buffer apply, created on first use.
rf_status host_streams(rf_plan_ *p)
{
    if (p->s_in) return RF_OK;
    cudaStream_t a = nullptr, b = nullptr;
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    rf_status s = cuda_status(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    if (s == RF_OK) s = cuda_status(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
    for (int k = 0; k < 3 && s == RF_OK; ++k)
        s = cuda_status(cudaEventCreateWithFlags(&e[k], cudaEventDisableTiming));
    if (s != RF_OK) {
        if (a) cudaStreamDestroy(a);
        if (b) cudaStreamDestroy(b);
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
        return s;
    }
    p->s_in = a;
    p->s_out = b;
    p->ev_in = e[0];
    p->ev_done = e[1];
    p->ev_out = e[2];
    return RF_OK;
}

constexpr int64_t kHostBatches = 12;
// With the streaming column kernel a launch's parallelism is columns x slice
// pairs and its serial chain of 2 ny steps sets a floor under each launch, so
// batches stay larger: on the regional workload 8 batches ran end to end at
// 34.1 Gpts/s against 32.0 with 4 and 17.8 with 12, whose launches outlast
// their copies.
constexpr int64_t kHostBatchesStream = 8;

// One domain through host buffers, pipelined over batches of levels: the
// copy in of a batch (stream s_in), its x and y launches (the caller's
// stream) and its copy out (stream s_out) overlap with the neighbouring
// batches'.  Each copy moves the batch's levels of all variables as one
// pitched 2-D copy (one row of nk levels per variable).
rf_status host_pipeline(rf_plan_ *p, Domain &D, const float *in, float *out, int nvar,
                        bool adjoint, cudaStream_t st)
{
    const int64_t nz = D.g.nz, plane = D.g.nx * D.g.ny;
    const int64_t n = (int64_t)nvar * nz * plane;
    RF_TRY(ensure(&D.stage, &D.stage_floats, n, &p->bytes));
    const int64_t nb = D.d[0].tcoef || D.d[1].tcoef ? kHostBatchesStream : kHostBatches;
    const int64_t nkb = (nz + nb - 1) / nb;
    int64_t nt = 0;   // scratch of the long-line kernel
    for (int dir = 0; dir < 2; ++dir)
        if (line_path(cfg_of(p, D, dir, nvar, nkb, adjoint)) ||
            line_path(cfg_of(p, D, dir, nvar, nz - (nz - 1) / nkb * nkb, adjoint)))
            nt = std::max(nt, D.d[dir].ntail * (int64_t)rec_floats(D.d[dir]));
    RF_TRY(ensure(&D.tscr, &D.tscr_floats, (int64_t)nvar * nz * nt, &p->bytes));
    const size_t pitch = (size_t)(nz * plane) * sizeof(float);
    const int K = p->opt.iters;
    // (a domain's stage is free here: every earlier host-buffer call ended
    // with its copies out complete, and nothing else uses the stage)
    for (int64_t k0 = 0; k0 < nz; k0 += nkb) {
        const int64_t nk = std::min(nkb, nz - k0);
        const size_t width = (size_t)(nk * plane) * sizeof(float);
        float *dev = D.stage + k0 * plane;
        RF_TRY(cuda_status(cudaMemcpy2DAsync(dev, pitch, in + k0 * plane, pitch, width,
                                             (size_t)nvar, cudaMemcpyHostToDevice, p->s_in)));
        RF_TRY(cuda_status(cudaEventRecord(p->ev_in, p->s_in)));
        RF_TRY(cuda_status(cudaStreamWaitEvent(st, p->ev_in, 0)));
        for (int pass = 0; pass < 2; ++pass) {
            const int dir = adjoint ? 1 - pass : pass;
            const Dir &q = D.d[dir];
            const LaunchCfg L = cfg_of(p, D, dir, nvar, nk, adjoint);
            if (p->opt.order == 3) {
                if (adjoint) launch_dir<3, true>(D, q, L, D.stage, D.stage, nvar, k0, nk, 1, st);
                else launch_dir<3, false>(D, q, L, D.stage, D.stage, nvar, k0, nk, 1, st);
            } else {
                if (adjoint) launch_dir<1, true>(D, q, L, D.stage, D.stage, nvar, k0, nk, K, st);
                else launch_dir<1, false>(D, q, L, D.stage, D.stage, nvar, k0, nk, K, st);
            }
            const rf_status s = cuda_status(cudaGetLastError());
            if (s != RF_OK) {
                if (p->sticky == RF_OK) p->sticky = s;
                return s;
            }
            ++p->launches;
        }
        RF_TRY(cuda_status(cudaEventRecord(p->ev_done, st)));
        RF_TRY(cuda_status(cudaStreamWaitEvent(p->s_out, p->ev_done, 0)));
        RF_TRY(cuda_status(cudaMemcpy2DAsync(out + k0 * plane, pitch, dev, pitch, width,
                                             (size_t)nvar, cudaMemcpyDeviceToHost, p->s_out)));
    }
    RF_TRY(cuda_status(cudaEventRecord(p->ev_out, p->s_out)));
    return cuda_status(cudaStreamWaitEvent(st, p->ev_out, 0));
}

rf_status tune_impl(rf_plan_ *p, int nvar, cudaStream_t st)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return RF_ECUDA;
    }
    const int64_t launches = p->launches;   // tuning launches are not counted
    rf_status s = RF_OK;
    for (Domain &D : p->dom) {
        const int64_t nf = (int64_t)nvar * D.g.nz * D.g.nx * D.g.ny;
        float *buf = nullptr;
        int64_t dummy = 0;
        s = dev_alloc(&buf, 2 * nf, &dummy);
        if (s != RF_OK) break;
        s = tune_domain(p, D, nvar, buf, nf, e0, e1, st);
        cudaStreamSynchronize(st);
        cudaFree(buf);
        if (s != RF_OK) break;
    }
    if (s == RF_OK && p->dom.size() > 1) s = tune_multi(p, nvar, e0, e1, st);
    p->launches = launches;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == RF_OK) s = cuda_status(cudaGetLastError());
    return s;
}

}  // namespace

extern "C" {

rf_status rf_options_default(rf_options *opt)
{
    if (!opt) return RF_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->order = 3;
    opt->iters = 1;
    opt->img_factor = 3.0;
    opt->norm = RF_NORM_GAUSS_PEAK;
    return RF_OK;
}

rf_status rf_coeffs(const rf_grid *grids, int ndomains, const uint8_t *const *mask,
                    const float *const *Lx, const float *const *Ly,
                    const rf_options *opt, void *stream, rf_plan *out)
{
    if (!grids || ndomains < 1 || !mask || !Lx || !Ly || !out) return RF_EINVAL;
    rf_options o;
    if (opt) o = *opt;
    else rf_options_default(&o);
    RF_TRY(check_options(o));
    for (int d = 0; d < ndomains; ++d) {
        RF_TRY(check_grid(grids[d]));
        if (!mask[d] || !Lx[d] || !Ly[d]) return RF_EINVAL;
    }
    rf_plan_ *P = new (std::nothrow) rf_plan_;
    if (!P) return RF_ENOMEM;
    P->opt = o;
    P->dom.resize((size_t)ndomains);
    cudaStream_t st = (cudaStream_t)stream;
    {
        rf_status s = dev_alloc(&P->dstatus, 1, &P->bytes);
        if (s == RF_OK) s = cuda_status(cudaMemsetAsync(P->dstatus, 0, sizeof(unsigned), st));
        if (s != RF_OK) {
            rf_plan_destroy(P);
            return s;
        }
    }
    for (int d = 0; d < ndomains; ++d) {
        P->dom[d].g = grids[d];
        P->dom[d].status = P->dstatus;
        P->dom[d].wait_polls = &P->wait_polls;
        rf_status s = build_domain(P, P->dom[d], mask[d], Lx[d], Ly[d], st);
        if (s != RF_OK) {
            rf_plan_destroy(P);
            return s;
        }
    }
    *out = P;
    return RF_OK;
}

rf_status rf_apply(rf_plan p, const float *const *in, float *const *out, int nvar,
                   void *stream)
{
    return apply_impl(p, in, out, nvar, false, (cudaStream_t)stream);
}

rf_status rf_apply_adjoint(rf_plan p, const float *const *in, float *const *out,
                           int nvar, void *stream)
{
    return apply_impl(p, in, out, nvar, true, (cudaStream_t)stream);
}

rf_status rf_apply_host(rf_plan p, const float *const *in, float *const *out,
                        int nvar, int adjoint, void *stream)
{
    if (!p || !in || !out || nvar < 1) return RF_EINVAL;
    for (size_t d = 0; d < p->dom.size(); ++d)
        if (!in[d] || !out[d]) return RF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    RF_TRY(host_streams(p));
    for (Domain &D : p->dom) {
        const size_t d = (size_t)(&D - p->dom.data());
        RF_TRY(host_pipeline(p, D, in[d], out[d], nvar, adjoint != 0, st));
    }
    return cuda_status(cudaStreamSynchronize(st));
}

}  // extern "C"

// ----------------------------------------------------------------------
// Allocation-free apply.  Its scratch (the anticausal start states of the
// segment ends) lives in one file-scope device array instead of memory the
// plan grows with cudaMalloc, so the call allocates nothing.  Every GPU that
// loads this library holds the array until the process exits.
namespace {

constexpr int64_t kStaticScratchFloats = (int64_t)1 << 21;   // 8 MiB
static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in for the address).
rf_status static_scratch(float **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return RF_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return RF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return RF_ECUDA;
        }
        g_static_ptr[dev] = static_cast<float *>(ptr);
    }
    *out = g_static_ptr[dev];
    return RF_OK;
}

}  // namespace

extern "C" {

rf_status rf_apply_static(rf_plan p, const float *const *in, float *const *out, int nvar,
                          int adjoint, void *stream)
{
    if (!p || !in || !out || nvar < 1) return RF_EINVAL;
    for (size_t d = 0; d < p->dom.size(); ++d) {
        if (!in[d] || !out[d]) return RF_EINVAL;
        const int64_t nslices = (int64_t)nvar * p->dom[d].g.nz;
        for (const Dir &q : p->dom[d].d)
            if (q.ntail > 0 && nslices * q.ntail * rec_floats(q) > kStaticScratchFloats)
                return RF_EINVAL;
    }
    float *scr = nullptr;
    RF_TRY(static_scratch(&scr));
    cudaStream_t st = (cudaStream_t)stream;
    const bool adj = adjoint != 0;
    for (size_t d = 0; d < p->dom.size(); ++d) {
        const Domain &D = p->dom[d];
        const int64_t nslices = (int64_t)nvar * D.g.nz;
        for (int pass = 0; pass < 2; ++pass) {
            const int dir = adj ? 1 - pass : pass;   // forward x then y
            const Dir &q = D.d[dir];
            LineArgs a{};
            a.in = pass == 0 ? in[d] : out[d];
            a.out = out[d];
            a.coef = q.coef;
            a.tail_base = q.tail_base;
            a.tmap = q.tmap;
            a.cvec = q.cst ? q.cvec : nullptr;
            a.nr = rec_floats(q);
            a.tscr = scr;
            a.kc = q.kc;
            a.carry = q.kc > 0 ? q.carry + (adj ? 2 * (q.kc - 1) * q.ntail : 0) : nullptr;
            a.n = q.n;
            a.nlines = q.nlines;
            a.pt_stride = q.pt_stride;
            a.line_stride = q.line_stride;
            a.plane = D.g.nx * D.g.ny;
            a.nz = D.g.nz;
            a.nvar = nvar;
            a.k0 = 0;
            a.nk = D.g.nz;
            a.ntail = q.ntail;
            a.ncl = D.ncl;
            a.iters = p->opt.order == 3 ? 1 : p->opt.iters;
            const unsigned blocks = (unsigned)((q.nlines * nslices + 127) / 128);
            if (p->opt.order == 3) {
                if (adj) line_kernel<3, true><<<blocks, 128, 0, st>>>(a);
                else line_kernel<3, false><<<blocks, 128, 0, st>>>(a);
            } else {
                if (adj) line_kernel<1, true><<<blocks, 128, 0, st>>>(a);
                else line_kernel<1, false><<<blocks, 128, 0, st>>>(a);
            }
            const rf_status s = cuda_status(cudaGetLastError());
            if (s != RF_OK) {
                if (p->sticky == RF_OK) p->sticky = s;
                return s;
            }
            ++p->launches;
        }
    }
    return RF_OK;
}

struct rf_graph_ {
    rf_plan plan = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;   // kernels per replay
};

rf_status rf_graph_create(rf_plan p, const float *const *in, float *const *out, int nvar,
                          int adjoint, rf_graph *g)
{
    if (!p || !in || !out || nvar < 1 || !g) return RF_EINVAL;
    *g = nullptr;
    const bool adj = adjoint != 0;
    // configurations and scratch first: the captured call must not allocate
    RF_TRY(apply_impl(p, in, out, nvar, adj, nullptr, true));
    cudaStream_t cs = nullptr;
    RF_TRY(cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)));
    const int64_t launches0 = p->launches;
    rf_status s = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    cudaGraph_t graph = nullptr;
    if (s == RF_OK) {
        s = apply_impl(p, in, out, nvar, adj, cs);
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (s == RF_OK) s = cuda_status(e);
    }
    cudaStreamDestroy(cs);
    const int64_t captured = p->launches - launches0;
    p->launches = launches0;   // counted when the graph runs
    cudaGraphExec_t exec = nullptr;
    if (s == RF_OK) s = cuda_status(cudaGraphInstantiate(&exec, graph, 0));
    rf_graph_ *G = s == RF_OK ? new (std::nothrow) rf_graph_ : nullptr;
    if (s == RF_OK && !G) s = RF_ENOMEM;
    if (s != RF_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    G->plan = p;
    G->graph = graph;
    G->exec = exec;
    G->launches = captured;
    *g = G;
    return RF_OK;
}

rf_status rf_graph_launch(rf_graph g, void *stream)
{
    if (!g) return RF_EINVAL;
    const rf_status s = cuda_status(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    if (s != RF_OK) {
        if (g->plan->sticky == RF_OK) g->plan->sticky = s;
        return s;
    }
    g->plan->launches += g->launches;
    return RF_OK;
}

rf_status rf_graph_destroy(rf_graph g)
{
    if (!g) return RF_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return RF_OK;
}

rf_status rf_plan_tune_batch(rf_plan p, int nvar, void *stream)
{
    if (!p || nvar < 1) return RF_EINVAL;
    if (p->dom.size() < 2) return RF_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return RF_ECUDA;
    }
    const int64_t launches = p->launches;
    rf_status s = tune_multi(p, nvar, e0, e1, (cudaStream_t)stream);
    p->launches = launches;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == RF_OK) s = cuda_status(cudaGetLastError());
    return s;
}

rf_status rf_plan_tune(rf_plan p, int nvar, void *stream)
{
    if (!p || nvar < 1) return RF_EINVAL;
    return tune_impl(p, nvar, (cudaStream_t)stream);
}

rf_status rf_plan_describe(rf_plan p, char *buf, size_t cap)
{
    if (!p || !buf || cap == 0) return RF_EINVAL;
    std::string t;
    char line[256];
    std::snprintf(line, sizeof line, "filter: order %d, K %d, img_factor %g, coasts %s%s\n",
                  p->opt.order, p->opt.iters, p->opt.img_factor,
                  plan_cst(p) ? "constant extension" : plan_carry(p) ? "carried across iterations" : "zero input",
                  (p->opt.flags & RF_FLAG_Q_CORRECTED) ? ", q-corrected" : "");
    t += line;
    for (size_t d = 0; d < p->dom.size(); ++d) {
        const Domain &D = p->dom[d];
        std::snprintf(line, sizeof line, "domain %zu: %lld x %lld x %lld, coefficient levels %lld\n", d,
                      (long long)D.g.nx, (long long)D.g.ny, (long long)D.g.nz, (long long)D.ncl);
        t += line;
        for (const auto &e : D.batch) {
            std::snprintf(line, sizeof line, "  nvar %lld: %lld levels per batch\n",
                          (long long)e.first, (long long)e.second);
            t += line;
        }
        for (int dir = 0; dir < 2; ++dir) {
            const Dir &q = D.d[dir];
            std::snprintf(line, sizeof line,
                          "  %s: lines %lld of %lld points, %d lanes per line, chunk %lld, segment ends %lld\n",
                          dir == 0 ? "x" : "y", (long long)q.nlines, (long long)q.n, q.P, (long long)q.C,
                          (long long)q.ntail);
            t += line;
            if (q.rsh.P > 0) {
                std::snprintf(line, sizeof line,
                              "    register kernel: chunk %d, %d lanes per line, record slots %d\n",
                              q.rsh.C, q.rsh.P, q.max_ends);
                t += line;
            }
            if (q.tcoef) t += "    streaming column kernel\n";
            for (const CfgEntry &e : q.cfgs) {
                if (e.cfg.strm)
                    std::snprintf(line, sizeof line, "    nvar %lld, %lld levels, %s: streaming kernel\n",
                                  (long long)e.nvar, (long long)e.nk, e.adjoint ? "adjoint" : "forward");
                else if (e.cfg.reg)
                    std::snprintf(line, sizeof line,
                                  "    nvar %lld, %lld levels, %s: register kernel C=%d P=%d smem=%zu "
                                  "CTAs/SM=%d\n",
                                  (long long)e.nvar, (long long)e.nk, e.adjoint ? "adjoint" : "forward",
                                  q.rsh.C, q.rsh.P, e.cfg.smem, e.cfg.occ);
                else if (e.cfg.tile)
                    std::snprintf(line, sizeof line,
                                  "    nvar %lld, %lld levels, %s: tile R=%d B=%d P=%d buffers=%d smem=%zu "
                                  "CTAs/SM=%d rows=%lld\n",
                                  (long long)e.nvar, (long long)e.nk, e.adjoint ? "adjoint" : "forward",
                                  e.cfg.sh.R, e.cfg.sh.B, e.cfg.sh.P, e.cfg.nbuf, e.cfg.smem, e.cfg.occ,
                                  (long long)e.cfg.groups);
                else
                    std::snprintf(line, sizeof line, "    nvar %lld, %lld levels, %s: line kernel\n",
                                  (long long)e.nvar, (long long)e.nk, e.adjoint ? "adjoint" : "forward");
                t += line;
            }
        }
    }
    for (const MultiCfg &c : p->mcfg) {
        if (c.occ == 0) continue;   // no domain of the pass has c.P lanes per line
        std::snprintf(line, sizeof line, "multi-domain %s %s, nvar %lld: R=%d B=%d P=%d smem=%zu CTAs/SM=%d\n",
                      c.dir == 0 ? "x" : "y", c.adjoint ? "adjoint" : "forward", (long long)c.nvar,
                      c.sh.R, c.sh.B, c.sh.P, c.smem, c.occ);
        t += line;
    }
    for (const auto &e : p->multi_pref) {
        std::snprintf(line, sizeof line, "nvar %lld: %s launches\n", (long long)e.first,
                      e.second ? "multi-domain" : "per-domain");
        t += line;
    }
    const size_t n = std::min(cap - 1, t.size());
    std::memcpy(buf, t.data(), n);
    buf[n] = '\0';
    return RF_OK;
}

rf_status rf_plan_set_wait_limit(rf_plan p, int polls)
{
    if (!p || polls < 0) return RF_EINVAL;
    p->wait_polls = polls;
    return RF_OK;
}

rf_status rf_plan_status(rf_plan p)
{
    if (!p) return RF_EINVAL;
    if (p->sticky == RF_OK && p->dstatus) {
        // the kernels' device-side status (a bounded wait that gave up)
        unsigned w = 0;
        if (cudaMemcpy(&w, p->dstatus, sizeof w, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            p->sticky = RF_ECUDA;
        } else if (w & 1u) {
            p->sticky = RF_ETIMEOUT;
        }
    }
    return p->sticky;
}

rf_status rf_plan_info(rf_plan p, int64_t *points_per_var, int *ndomains,
                       int64_t *device_bytes, int64_t *launches)
{
    if (!p) return RF_EINVAL;
    int64_t pts = 0;
    for (auto &d : p->dom) pts += d.g.nx * d.g.ny * d.g.nz;
    if (points_per_var) *points_per_var = pts;
    if (ndomains) *ndomains = (int)p->dom.size();
    if (device_bytes) *device_bytes = p->bytes;
    if (launches) *launches = p->launches;
    return RF_OK;
}

rf_status rf_plan_destroy(rf_plan p)
{
    if (!p) return RF_OK;
    cudaDeviceSynchronize();
    free_plan(p);
    delete p;
    return RF_OK;
}

const char *rf_status_string(rf_status s)
{
    switch (s) {
    case RF_OK: return "RF_OK";
    case RF_EINVAL: return "RF_EINVAL: invalid argument";
    case RF_ENOMEM: return "RF_ENOMEM: out of memory";
    case RF_ECUDA: return "RF_ECUDA: CUDA error";
    case RF_ETIMEOUT: return "RF_ETIMEOUT: device-side wait timed out";
    case RF_EUNSUPPORTED: return "RF_EUNSUPPORTED: not supported";
    }
    return "unknown rf_status";
}

}  // extern "C"
