/*
 * rfvh.h -- C ABI of the GB300 recursive-filter library for the horizontal
 * background-error covariance operator V_H of an ocean 3D-VAR.
 *
 * Method: Farina, Dobricic, Storto, Masina, Cuomo, "A Revised Scheme to
 * Compute Horizontal Covariances in an Oceanographic 3D-VAR Assimilation
 * System" (arXiv 1404.5756).  V_H = G_y G_x (Sec. 2.2): a 1-D recursive
 * filter is applied along every row (x) and then along every column (y) of
 * every level of every variable.  Each 1-D filter is a causal (forward) pass
 * followed by an anticausal (backward) pass (Sec. 3, Eqs. "one1"/"two2"):
 *   - order 3: the third-order filter of Theorem 3.1, one iteration, with
 *     per-point coefficients from sigma_i = R_i/dx_i;
 *   - order 1: the first-order filter of Sec. 3.1 iterated K times, with the
 *     coefficients of Hayden's relation (Eq. "crucial").
 * Initial conditions are the heuristic zero-state ones of Sec. 3.1.  Coasts
 * use imaginary sea points (Sec. 1, Sec. 4): each run of sea points of a
 * line is extended at both ends by n_img = ceil(img_factor * sigma_coast)
 * points of zero input carrying the coastal point's coefficients; only the
 * sea points are written.  Land points are written as 0 and their input is
 * ignored.  rf_apply_adjoint applies V_H^T = G_x^T G_y^T (the transpose the
 * 3D-VAR gradient of Eq. "eight" needs).
 *
 * Conventions for every call:
 *   - Fields are FP32, laid out [nvar][nz][ny][nx] with x fastest, one
 *     contiguous array per domain, in device memory.
 *   - Masks are uint8 [mask_nz][ny][nx] (nonzero = sea); length scales are
 *     FP32 [L_nz][ny][nx] in grid units (sigma = R/dx).  mask_nz and L_nz
 *     are 1 (one 2-D field shared by every level) or nz.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Apply calls are asynchronous on it; rf_coeffs synchronises it.
 *   - No call throws; every call returns an rf_status.  Argument errors are
 *     reported synchronously, before any GPU work is queued.
 *   - The caller owns every buffer it passes in; the plan owns every buffer
 *     it derives (coefficients, boundary maps, work lists, scratch).
 */
#ifndef RFVH_H
#define RFVH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RF_OK = 0,
    RF_EINVAL = 1,        /* bad argument: null pointer, size, option, length scale */
    RF_ENOMEM = 2,        /* device or host allocation failed */
    RF_ECUDA = 3,         /* a CUDA call or kernel launch failed */
    RF_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    RF_EUNSUPPORTED = 5   /* valid request this build does not provide */
} rf_status;

enum {
    RF_NORM_GAUSS_PEAK = 0, /* Theorem 3.1 normalisation: impulse response peaks
                               near 1, sums to sqrt(2 pi) sigma per direction;
                               the 1st-RF gets (2 pi sigma^2)^(1/(4K)) per pass */
    RF_NORM_UNIT_SUM = 1    /* every pass has DC gain 1 (the literal 1st-RF) */
};

/* rf_options.flags.  RF_FLAG_Q_CORRECTED (order 3 only, not the paper's
 * filter): the Theorem 3.1 coefficients are taken at the scale q whose
 * impulse-response variance, 2 (P1/P0) q + 2 ((P1/P0)^2 - 2 P2/P0) q^2, equals
 * sigma^2, so the filter's variance is sigma^2 instead of about
 * 3.10 sigma + 1.18 sigma^2; the normalisation stays that of sigma (DC gain
 * sqrt(2 pi) sigma per direction).  The number of imaginary points still
 * follows sigma.
 *
 * RF_FLAG_COAST_CONSTANT (either order, not the paper's coasts): the
 * imaginary sea points at each end of a sea segment carry the segment's edge
 * value (its first sea value on the left, its last on the right) instead of
 * zero -- one of the other coastal boundary conditions the Conclusions leave
 * for future work.  The adjoint is the exact transpose: the adjoint values
 * at the imaginary points are added to the edge point they copied.  With
 * img_factor = 0 (no imaginary points) it changes nothing.
 *
 * RF_FLAG_COAST_CARRIED (not the paper's coasts; another of the conditions
 * the Conclusions leave open): for the 1st-RF with K > 1 iterations the
 * imaginary points start at zero and keep, from one iteration to the next,
 * the values the filter left in them, i.e. each line segment is extended
 * once, filtered K times and read back once (R G_ext^K R^T instead of
 * (R G_ext R^T)^K); the adjoint is R (G_ext^T)^K R^T.  For K = 1, the 3rd-RF
 * or img_factor = 0 it changes nothing.  It excludes RF_FLAG_COAST_CONSTANT
 * (RF_EINVAL).  Flags combine with |. */
enum { RF_FLAG_Q_CORRECTED = 1, RF_FLAG_COAST_CONSTANT = 2, RF_FLAG_COAST_CARRIED = 4 };

typedef struct rf_plan_ *rf_plan;
typedef struct rf_graph_ *rf_graph;

/* One domain's grid. */
typedef struct {
    int64_t nx, ny, nz;   /* points along x (contiguous), y, and levels     */
    int64_t mask_nz;      /* 1 or nz                                        */
    int64_t L_nz;         /* 1 or nz                                        */
} rf_grid;

typedef struct {
    int order;            /* 3 (Theorem 3.1) or 1 (Sec. 3.1)                 */
    int iters;            /* K: must be 1 for order 3, >= 1 for order 1      */
    double img_factor;    /* imaginary points per coast end = ceil(img_factor
                             * sigma_coast); 0 = the bare heuristic ICs;
                             +INFINITY = the infinite imaginary sea (the
                             closed-form limit of the boundary map, zero-input
                             coasts only: with RF_FLAG_COAST_CONSTANT it gives
                             RF_EUNSUPPORTED); must be >= 0, not NaN          */
    int norm;             /* RF_NORM_GAUSS_PEAK or RF_NORM_UNIT_SUM          */
    int flags;            /* RF_FLAG_Q_CORRECTED (order 3 only) |
                             RF_FLAG_COAST_CONSTANT or RF_FLAG_COAST_CARRIED,
                             or 0                                            */
    int chunk;            /* chunk-length override: must be 0 (automatic);
                             any other value gives RF_EUNSUPPORTED, since the
                             kernels derive the chunking from the line length */
    int tile;             /* tile-shape override: must be 0 (automatic, or the
                             autotuner's choice); other values give
                             RF_EUNSUPPORTED                                  */
} rf_options;

/* Fill *opt with the defaults: order 3, iters 1, img_factor 3, Gaussian-peak
 * normalisation.  Returns RF_EINVAL if opt is NULL. */
rf_status rf_options_default(rf_options *opt);

/* Build a plan for `ndomains` independent domains (a ragged batch).
 *   grids[d]          grid of domain d (host array of ndomains structs)
 *   mask[d]           device pointer, uint8 [mask_nz][ny][nx], nonzero = sea
 *   Lx[d], Ly[d]      device pointers, FP32 [L_nz][ny][nx], length scale
 *                     along x and along y in grid units; must be finite and
 *                     > 0 wherever the point is sea on some level
 *   opt               options (host); NULL means rf_options_default
 *   stream            cudaStream_t used for the set-up work; synchronised
 *   out               receives the plan; untouched on error
 * Computes the per-point coefficients of Theorem 3.1 (order 3) or of Sec.
 * 3.1 (order 1) in FP64 on the GPU and stores them as FP32, finds the sea
 * segments of every line and computes, in FP64, the map that takes the
 * forward state at each segment's last sea point to the backward start state
 * (the effect of the n_img imaginary points).  The caller's mask and length
 * scale buffers may be freed once the call returns.
 * The map of the infinite imaginary sea (img_factor = +INFINITY) is the
 * limit sum_{j>=0} A^j Q A^j of the finite one, solved in FP64 as its Stein
 * equation M = Q + A M A.
 * Errors: RF_EINVAL (null pointers, ndomains < 1, nx/ny/nz < 1, mask_nz or
 * L_nz not in {1, nz}, bad options, invalid length scale at a sea point),
 * RF_EUNSUPPORTED (non-zero chunk or tile override; infinite imaginary sea
 * with constant-extension coasts), RF_ENOMEM, RF_ECUDA. */
rf_status rf_coeffs(const rf_grid *grids, int ndomains,
                    const uint8_t *const *mask, const float *const *Lx,
                    const float *const *Ly, const rf_options *opt,
                    void *stream, rf_plan *out);

/* out = V_H in, i.e. G_y G_x on every level of every variable of every
 * domain (Sec. 2.2; G_x, G_y per Theorem 3.1 or Sec. 3.1 and the plan's
 * options).
 *   in[d], out[d]     device pointers to domain d's FP32 field
 *                     [nvar][nz][ny][nx]; in[d] == out[d] is allowed;
 *                     distinct domains must not overlap
 *   nvar              variables per domain (e.g. 2 for T and S), >= 1
 * With several domains the x pass of all domains is one persistent launch
 * over a work list of (domain, line block, slice group) items, then the y
 * pass likewise (per 32 domains), unless rf_plan_tune found separate
 * per-domain launches faster.
 * Asynchronous on `stream`.  Errors: RF_EINVAL (null plan or pointers,
 * nvar < 1), RF_ENOMEM (scratch growth), RF_ECUDA (launch failure). */
rf_status rf_apply(rf_plan p, const float *const *in, float *const *out,
                   int nvar, void *stream);

/* out = V_H^T in = G_x^T G_y^T in: the exact transpose of rf_apply (the
 * transposed recursions of each pass, the y direction first).  Same
 * arguments, ownership and errors as rf_apply. */
rf_status rf_apply_adjoint(rf_plan p, const float *const *in,
                           float *const *out, int nvar, void *stream);

/* End-to-end variant of rf_apply / rf_apply_adjoint on HOST buffers: copies
 * in[d] (host, ideally pinned) to plan-owned device staging, applies V_H
 * (adjoint != 0: V_H^T), copies the result back into out[d] (host) and
 * synchronises `stream`.  Per domain the work is pipelined over up to 12
 * batches of levels: the copy in of one batch, the filtering of the one
 * before and the copy out of the one before that overlap (two plan-owned
 * copy streams; the kernels run on `stream`).  in[d] and out[d] may be the
 * same buffer.  The staging buffers and copy streams are created on first
 * use and kept by the plan.  Errors as rf_apply. */
rf_status rf_apply_host(rf_plan p, const float *const *in, float *const *out,
                        int nvar, int adjoint, void *stream);

/* Allocation-free variant of rf_apply / rf_apply_adjoint (adjoint != 0),
 * for callers that must not allocate device memory at the time they apply
 * the operator: code that runs inside a framework which owns every device
 * allocation through its own pool, code that must not trigger the implicit
 * synchronisation of cudaMalloc/cudaFree, or real-time loops that may not
 * allocate after start-up.  The paper has no counterpart; it is a service of
 * this library.  It runs the one-thread-per-line kernel for both directions
 * and keeps the per-call scratch (per segment end of every slice the
 * anticausal start state, r floats: 3; 4 with RF_FLAG_COAST_CONSTANT; 2 + 2K
 * with RF_FLAG_COAST_CARRIED) in one static device array of 2^21 floats
 * (8 MiB) inside the library, which every GPU that loads the library holds
 * until the process exits.  The call itself performs no device allocation;
 * the plan (built earlier by rf_coeffs) must exist.
 *   in[d], out[d], nvar, stream   as rf_apply
 * Limit: for every domain and direction, nvar * nz * (segment ends of that
 * direction) * r must not exceed 2^21, else RF_EINVAL before any launch.
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call outside any stream capture.  The kept address does not survive
 * cudaDeviceReset (or any other teardown of the device's primary context):
 * after one, the plans are invalid anyway, and this call must not be used
 * again in the same process.
 * Every call uses the same array: calls that overlap on the GPU (other
 * streams, other threads, other plans) race and give wrong results.  Each
 * call writes every scratch entry it reads, so no clearing is needed.
 * Errors: RF_EINVAL, RF_ECUDA, RF_EUNSUPPORTED (device index >= 64). */
rf_status rf_apply_static(rf_plan p, const float *const *in, float *const *out,
                          int nvar, int adjoint, void *stream);

/* Launch-shape autotuner.  For `nvar` variables per domain, times every
 * shape the tile kernel is built for (lines per CTA, slices per thread,
 * single or double buffering) that fits shared memory, for the forward and
 * the adjoint operator in each direction of each domain, on plan-owned
 * scratch fields (allocated for the call and freed before it returns), and
 * keeps the fastest for later rf_apply / rf_apply_adjoint calls with the same
 * nvar.  Without tuning a fixed rule picks the shape.  Synchronises `stream`.
 * Errors: RF_EINVAL (null plan, nvar < 1), RF_ENOMEM, RF_ECUDA. */
rf_status rf_plan_tune(rf_plan p, int nvar, void *stream);

/* The multi-domain part of rf_plan_tune alone, for plans of many domains
 * where tuning every domain separately would take long: times every shape
 * of the multi-domain launch of each pass (forward and adjoint) and then
 * whole applications with multi-domain against per-domain launches, keeping
 * the faster for later calls with the same nvar.  Allocates scratch fields
 * for all domains at once for the call.  A plan of one domain: no-op.
 * Synchronises `stream`.  Errors: as rf_plan_tune. */
rf_status rf_plan_tune_batch(rf_plan p, int nvar, void *stream);

/* CUDA graph of one application: captures rf_apply (adjoint == 0) or
 * rf_apply_adjoint (adjoint != 0) of the given buffers and nvar into an
 * executable graph, so a loop that applies the operator many times (a
 * minimisation) pays one graph launch per application.
 *   in[d], out[d], nvar   as rf_apply; the graph keeps these pointers, so
 *                         the buffers must outlive it
 *   g                     receives the graph; untouched on error
 * Chooses launch shapes and grows the plan's scratch before capturing, so
 * the captured call allocates nothing; the capture runs on a private stream
 * and launches nothing.  Call rf_plan_tune first if tuned shapes are wanted:
 * later tuning does not change an existing graph.  The graph uses the plan's
 * buffers: destroy graphs before their plan, and do not replay a graph
 * concurrently with another use of the same plan.
 * Errors: RF_EINVAL, RF_ENOMEM, RF_ECUDA. */
rf_status rf_graph_create(rf_plan p, const float *const *in, float *const *out,
                          int nvar, int adjoint, rf_graph *g);

/* Replays the graph on `stream` (asynchronous).  Errors: RF_EINVAL (null
 * graph), RF_ECUDA. */
rf_status rf_graph_launch(rf_graph g, void *stream);

/* Frees the graph (after the work it launched has finished).  NULL is
 * accepted. */
rf_status rf_graph_destroy(rf_graph g);

/* Text description of the plan (domains, chunking, the launch
 * configurations chosen so far per variable count, level batch and
 * direction, multi-domain shapes) into buf, at most cap - 1 characters plus
 * a terminating NUL (truncated if longer).  Errors: RF_EINVAL (null plan or
 * buffer, cap == 0). */
rf_status rf_plan_describe(rf_plan p, char *buf, size_t cap);

/* Sticky status of the plan: RF_OK, or the first error a launch or a
 * device-side check recorded since the plan was built.  RF_ETIMEOUT: a
 * kernel's bounded wait on an asynchronous copy gave up (the kernel recorded
 * it, let the copy land and returned without filtering its part; the
 * context stays usable). */
rf_status rf_plan_status(rf_plan p);

/* Bound of the kernels' device-side waits for this plan's later launches,
 * in polls of the waiting mbarrier (each poll may suspend the thread for a
 * short, system-dependent time).  rf_coeffs sets 2^20, far above any real
 * copy time; 0 makes every such wait give up at once, which is how the
 * timeout path (RF_ETIMEOUT from rf_plan_status) is tested without stalling
 * or faulting a GPU.  The paper has no counterpart.  Errors: RF_EINVAL (null
 * plan, polls < 0). */
rf_status rf_plan_set_wait_limit(rf_plan p, int polls);

/* Counts of the plan: total grid points per variable over all domains
 * (nx*ny*nz summed), number of domains, device bytes owned by the plan, and
 * the number of kernels the apply calls have launched since the plan was
 * built.  Any output pointer may be NULL. */
rf_status rf_plan_info(rf_plan p, int64_t *points_per_var, int *ndomains,
                       int64_t *device_bytes, int64_t *launches);

/* Free everything the plan owns (waits for the device first).  NULL is a
 * no-op returning RF_OK. */
rf_status rf_plan_destroy(rf_plan p);

/* Static human-readable name of a status code. */
const char *rf_status_string(rf_status s);

#ifdef __cplusplus
}
#endif

#endif /* RFVH_H */
