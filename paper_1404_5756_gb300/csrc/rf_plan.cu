// rf_plan.cu -- C ABI of the recursive-filter library: plan construction
// (validation, sea segments, FP64 coefficients and boundary maps) and the
// apply entry points.  See include/rfvh.h for the contract of every call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "rfvh.h"
#include "rf_coef.cuh"
#include "rf_line.cuh"

using namespace rfvh;

namespace {

struct TailSpec {
    float sigma;
    int n_img;
};

struct Domain {
    rf_grid g{};
    int64_t ncl = 1;                 // levels of distinct segment structure
    uint8_t *mask = nullptr;         // [mask_nz][ny][nx]
    float4 *coef_x = nullptr;        // [L_nz][ny][nx]
    float4 *coef_y = nullptr;
    int32_t *tail_x = nullptr;       // [ncl][ny][nx]
    int32_t *tail_y = nullptr;
    double *tmap_x = nullptr;        // [ntail_x][9]
    double *tmap_y = nullptr;
    int64_t ntail_x = 0, ntail_y = 0;
    float *yscr = nullptr;           // backward start states
    int64_t yscr_floats = 0;
    float *stage = nullptr;          // host-API staging
    int64_t stage_floats = 0;
};

}  // namespace

struct rf_plan_ {
    rf_options opt{};
    std::vector<Domain> dom;
    int64_t bytes = 0;
    int64_t launches = 0;
    rf_status sticky = RF_OK;
};

namespace {

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
    cudaFree(d.mask);
    cudaFree(d.coef_x);
    cudaFree(d.coef_y);
    cudaFree(d.tail_x);
    cudaFree(d.tail_y);
    cudaFree(d.tmap_x);
    cudaFree(d.tmap_y);
    cudaFree(d.yscr);
    cudaFree(d.stage);
    d = Domain{};
}

rf_status check_options(const rf_options &o)
{
    if (o.order != 1 && o.order != 3) return RF_EINVAL;
    if (o.iters < 1 || (o.order == 3 && o.iters != 1)) return RF_EINVAL;
    if (!(o.img_factor >= 0.0) || !std::isfinite(o.img_factor)) return RF_EINVAL;
    if (o.norm != RF_NORM_GAUSS_PEAK && o.norm != RF_NORM_UNIT_SUM) return RF_EINVAL;
    if (o.flags != 0 || o.chunk < 0 || o.tile < 0) return RF_EINVAL;
    return RF_OK;
}

rf_status check_grid(const rf_grid &g)
{
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return RF_EINVAL;
    if (!(g.mask_nz == 1 || g.mask_nz == g.nz)) return RF_EINVAL;
    if (!(g.L_nz == 1 || g.L_nz == g.nz)) return RF_EINVAL;
    // indices inside the kernels are 64-bit, but a line index times the
    // slice count must stay well inside int64 and lines inside int32 counts
    if (g.nx > (1 << 30) || g.ny > (1 << 30) || g.nz > (1 << 20)) return RF_EINVAL;
    return RF_OK;
}

// FP64 coefficients on the device, stored as FP32 (beta, e, c1, c2).
__global__ void coef_kernel(int64_t n, const float *__restrict__ L,
                            float4 *__restrict__ coef, int order, int K, int norm)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = (double)L[i];
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s > 0.0 && isfinite(s)) {
        Coef64 c = coef_fp64(s, order, K, norm);
        r = make_float4((float)c.beta, (float)c.e, (float)c.c1, (float)c.c2);
    }
    coef[i] = r;
}

__global__ void tail_kernel(int64_t n, const TailSpec *__restrict__ spec,
                            double *__restrict__ tmap, int order, int K, int norm)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    tail_map_fp64((double)spec[i].sigma, spec[i].n_img, order, K, norm, tmap + 9 * i);
}

int n_imaginary(double img_factor, float sigma)
{
    if (!(img_factor > 0.0)) return 0;
    return (int)std::ceil(img_factor * (double)sigma);
}

// Host analysis of one domain: validate length scales at sea points, find
// the last sea point of every segment of every line, give each one a
// boundary-map index and record its coastal sigma and imaginary count.
rf_status analyse(const rf_grid &g, int64_t ncl, const std::vector<uint8_t> &mask,
                  const std::vector<float> &Lx, const std::vector<float> &Ly,
                  double img_factor, std::vector<int32_t> &tx,
                  std::vector<int32_t> &ty, std::vector<TailSpec> &sx,
                  std::vector<TailSpec> &sy)
{
    const int64_t nx = g.nx, ny = g.ny, plane = nx * ny;
    tx.assign((size_t)(ncl * plane), -1);
    ty.assign((size_t)(ncl * plane), -1);
    for (int64_t k = 0; k < ncl; ++k) {
        const uint8_t *m = mask.data() + (g.mask_nz > 1 ? k : 0) * plane;
        const float *lx = Lx.data() + (g.L_nz > 1 ? k : 0) * plane;
        const float *ly = Ly.data() + (g.L_nz > 1 ? k : 0) * plane;
        for (int64_t p = 0; p < plane; ++p) {
            if (!m[p]) continue;
            if (!(lx[p] > 0.f) || !std::isfinite(lx[p])) return RF_EINVAL;
            if (!(ly[p] > 0.f) || !std::isfinite(ly[p])) return RF_EINVAL;
        }
        if (!(img_factor > 0.0)) continue;
        int32_t *txk = tx.data() + k * plane;
        int32_t *tyk = ty.data() + k * plane;
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = j * nx + i;
                if (!m[p]) continue;
                if (i == nx - 1 || !m[p + 1]) {
                    if (sx.size() >= (size_t)INT32_MAX) return RF_EINVAL;
                    txk[p] = (int32_t)sx.size();
                    sx.push_back({lx[p], n_imaginary(img_factor, lx[p])});
                }
                if (j == ny - 1 || !m[p + nx]) {
                    if (sy.size() >= (size_t)INT32_MAX) return RF_EINVAL;
                    tyk[p] = (int32_t)sy.size();
                    sy.push_back({ly[p], n_imaginary(img_factor, ly[p])});
                }
            }
    }
    return RF_OK;
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

rf_status build_domain(rf_plan_ *P, Domain &d, const uint8_t *mask_dev,
                       const float *Lx_dev, const float *Ly_dev, cudaStream_t st)
{
    const rf_grid &g = d.g;
    const int64_t plane = g.nx * g.ny;
    const int64_t ncl = (g.mask_nz > 1 || g.L_nz > 1) ? g.nz : 1;
    d.ncl = ncl;
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

    std::vector<int32_t> tx, ty;
    std::vector<TailSpec> sx, sy;
    RF_TRY(analyse(g, ncl, hm, hx, hy, P->opt.img_factor, tx, ty, sx, sy));
    d.ntail_x = (int64_t)sx.size();
    d.ntail_y = (int64_t)sy.size();

    RF_TRY(dev_alloc(&d.mask, g.mask_nz * plane, &P->bytes));
    RF_TRY(dev_alloc(&d.coef_x, g.L_nz * plane, &P->bytes));
    RF_TRY(dev_alloc(&d.coef_y, g.L_nz * plane, &P->bytes));
    RF_TRY(dev_alloc(&d.tail_x, ncl * plane, &P->bytes));
    RF_TRY(dev_alloc(&d.tail_y, ncl * plane, &P->bytes));
    RF_TRY(dev_alloc(&d.tmap_x, 9 * d.ntail_x, &P->bytes));
    RF_TRY(dev_alloc(&d.tmap_y, 9 * d.ntail_y, &P->bytes));

    RF_TRY(cuda_status(cudaMemcpyAsync(d.mask, hm.data(), hm.size(),
                                       cudaMemcpyHostToDevice, st)));
    RF_TRY(cuda_status(cudaMemcpyAsync(d.tail_x, tx.data(), tx.size() * 4,
                                       cudaMemcpyHostToDevice, st)));
    RF_TRY(cuda_status(cudaMemcpyAsync(d.tail_y, ty.data(), ty.size() * 4,
                                       cudaMemcpyHostToDevice, st)));

    const int o = P->opt.order, K = P->opt.iters, nm = P->opt.norm;
    const int64_t nl = g.L_nz * plane;
    const int blk = 256;
    coef_kernel<<<(unsigned)((nl + blk - 1) / blk), blk, 0, st>>>(nl, Lx_dev, d.coef_x, o, K, nm);
    coef_kernel<<<(unsigned)((nl + blk - 1) / blk), blk, 0, st>>>(nl, Ly_dev, d.coef_y, o, K, nm);
    RF_TRY(cuda_status(cudaGetLastError()));

    for (int dir = 0; dir < 2; ++dir) {
        const std::vector<TailSpec> &sp = dir == 0 ? sx : sy;
        double *tm = dir == 0 ? d.tmap_x : d.tmap_y;
        if (sp.empty()) continue;
        TailSpec *dsp = nullptr;
        int64_t dummy = 0;
        RF_TRY(dev_alloc(&dsp, (int64_t)sp.size(), &dummy));
        rf_status s = cuda_status(cudaMemcpyAsync(dsp, sp.data(), sp.size() * sizeof(TailSpec),
                                                  cudaMemcpyHostToDevice, st));
        if (s == RF_OK) {
            int64_t n = (int64_t)sp.size();
            tail_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, dsp, tm, o, K, nm);
            s = cuda_status(cudaGetLastError());
        }
        if (s == RF_OK) s = cuda_status(cudaStreamSynchronize(st));
        cudaFree(dsp);
        RF_TRY(s);
    }
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

template <int ORDER, bool ADJ>
void launch_pass(const LineArgs &a, cudaStream_t st)
{
    const int64_t nlines = a.along_x ? a.ny : a.nx;
    const int64_t threads = nlines * a.nslices;
    line_kernel<ORDER, ADJ><<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(a);
}

rf_status apply_impl(rf_plan p, const float *const *in, float *const *out,
                     int nvar, bool adjoint, cudaStream_t st)
{
    if (!p || !in || !out || nvar < 1) return RF_EINVAL;
    for (size_t d = 0; d < p->dom.size(); ++d)
        if (!in[d] || !out[d]) return RF_EINVAL;
    for (size_t d = 0; d < p->dom.size(); ++d) {
        Domain &D = p->dom[d];
        const int64_t nslices = (int64_t)nvar * D.g.nz;
        const int64_t nt = D.ntail_x > D.ntail_y ? D.ntail_x : D.ntail_y;
        rf_status s = ensure(&D.yscr, &D.yscr_floats, nslices * nt * 3, &p->bytes);
        if (s != RF_OK) return s;
        LineArgs a{};
        a.mask = D.mask;
        a.yscr = D.yscr;
        a.nx = D.g.nx;
        a.ny = D.g.ny;
        a.nz = D.g.nz;
        a.nslices = nslices;
        a.mask_nz = (int)D.g.mask_nz;
        a.L_nz = (int)D.g.L_nz;
        a.ncl = (int)D.ncl;
        a.iters = p->opt.iters;
        for (int pass = 0; pass < 2; ++pass) {
            const bool along_x = adjoint ? pass == 1 : pass == 0;
            a.in = pass == 0 ? in[d] : out[d];
            a.out = out[d];
            a.along_x = along_x ? 1 : 0;
            a.coef = along_x ? D.coef_x : D.coef_y;
            a.tail = along_x ? D.tail_x : D.tail_y;
            a.tmap = along_x ? D.tmap_x : D.tmap_y;
            a.ntail = along_x ? D.ntail_x : D.ntail_y;
            if (p->opt.order == 3) {
                if (adjoint) launch_pass<3, true>(a, st);
                else launch_pass<3, false>(a, st);
            } else {
                if (adjoint) launch_pass<1, true>(a, st);
                else launch_pass<1, false>(a, st);
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
    for (int d = 0; d < ndomains; ++d) {
        P->dom[d].g = grids[d];
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
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nd = p->dom.size();
    std::vector<const float *> din(nd);
    std::vector<float *> dout(nd);
    for (size_t d = 0; d < nd; ++d) {
        Domain &D = p->dom[d];
        if (!in[d] || !out[d]) return RF_EINVAL;
        const int64_t n = (int64_t)nvar * D.g.nz * D.g.ny * D.g.nx;
        RF_TRY(ensure(&D.stage, &D.stage_floats, n, &p->bytes));
        RF_TRY(cuda_status(cudaMemcpyAsync(D.stage, in[d], (size_t)n * 4,
                                           cudaMemcpyHostToDevice, st)));
        din[d] = D.stage;
        dout[d] = D.stage;
    }
    RF_TRY(apply_impl(p, din.data(), dout.data(), nvar, adjoint != 0, st));
    for (size_t d = 0; d < nd; ++d) {
        Domain &D = p->dom[d];
        const int64_t n = (int64_t)nvar * D.g.nz * D.g.ny * D.g.nx;
        RF_TRY(cuda_status(cudaMemcpyAsync(out[d], D.stage, (size_t)n * 4,
                                           cudaMemcpyDeviceToHost, st)));
    }
    return cuda_status(cudaStreamSynchronize(st));
}

rf_status rf_plan_status(rf_plan p)
{
    if (!p) return RF_EINVAL;
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
    for (auto &d : p->dom) free_domain(d);
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
