"""Constant-extension coasts (RF_FLAG_COAST_CONSTANT): the imaginary sea
points carry the segment's edge values instead of zero, one of the other
coastal boundary conditions the paper's Conclusions leave for future work.
Parity with the FP64 oracle's constant extension (bar 1e-5 of max |oracle|),
through both tile-kernel widths (16 and 32 lanes per line, 64- and 128-bit
segment masks), the long-line kernel, the multi-domain launch and the
allocation-free entry point; the GPU dot test; and the properties that hold
at any size (img_factor 0 changes nothing; a constant field keeps its gain
up to the coast)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Options, Plan, _lib, synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
FILTERS = [(3, 1), (1, 5)]


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def opts(order, K, img=3.0, coast="constant", **kw):
    return Options(order=order, iters=K, img_factor=img, coast=coast, **kw)


def gpu(mask, Lx, Ly, x, order, K, adjoint=False, img=3.0, coast="constant", **kw):
    plan = Plan(dict(mask=mask, Lx=Lx, Ly=Ly, nz=x.shape[1]), opts(order, K, img, coast, **kw))
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    y = plan.apply_adjoint(xt) if adjoint else plan.apply(xt)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return y.cpu().numpy()


def oracle(mask, Lx, Ly, x, order, K, adjoint=False, img=3.0, qcorr=False):
    return orc.vh(np.asarray(x, np.float64), mask, np.asarray(Lx, np.float64),
                  np.asarray(Ly, np.float64), order=order, iters=K, adjoint=adjoint,
                  img_factor=img, qcorr=qcorr, coast=orc.COAST_CONSTANT)


def random_case(seed, ny, nx, nz=2, nvar=2, land=0.25, lo=1.0, hi=12.0):
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=(ny, nx)) > land).astype(np.uint8)
    Lx = rng.uniform(lo, hi, (ny, nx)).astype(np.float32)
    Ly = rng.uniform(lo, hi, (ny, nx)).astype(np.float32)
    x = rng.standard_normal((nvar, nz, ny, nx)).astype(np.float32)
    return mask, Lx, Ly, x


@pytest.fixture(scope="module")
def regional():
    w = synth.workload(2, nz=2, nvar=2)
    return w["mask"], w["Lx"], w["Ly"], w["x"]


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_regional_grid_matches_oracle(regional, order, K, adjoint):
    """1024 x 384 with coastlines: rows on 32 lanes, columns on 16 (3rd-RF)."""
    mask, Lx, Ly, x = regional
    g = gpu(mask, Lx, Ly, x, order, K, adjoint)
    o = oracle(mask, Lx, Ly, x, order, K, adjoint)
    assert rel_err(g, o) <= TOL
    # the option changes the result near the coasts
    z = gpu(mask, Lx, Ly, x, order, K, adjoint, coast="zero")
    assert rel_err(z, o) > 1e-3


EDGE_GRIDS = [(1, 1), (1, 7), (9, 1), (3, 5), (17, 13), (33, 65), (130, 3)]


@pytest.mark.parametrize("ny,nx", EDGE_GRIDS)
@pytest.mark.parametrize("order,K", FILTERS)
def test_small_and_ragged_grids(ny, nx, order, K):
    """Grid-edge segment starts, one-point segments and chunks past the
    line's end."""
    mask, Lx, Ly, x = random_case(ny * 100 + nx, ny, nx, land=0.3, lo=0.5)
    for adjoint in (False, True):
        g = gpu(mask, Lx, Ly, x, order, K, adjoint)
        o = oracle(mask, Lx, Ly, x, order, K, adjoint)
        if np.abs(o).max() == 0:
            assert np.all(g == 0)
        else:
            assert rel_err(g, o) <= TOL, adjoint


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("nx", [300, 1500, 3000, 4200])
def test_line_lengths_across_kernels(order, K, nx):
    """Rows of 300 points (16 lanes for the 3rd-RF), 1500 (32 lanes, 64-bit
    masks), 3000 (95-point chunks, 128-bit masks) and 4200 (the long-line
    kernel)."""
    mask, Lx, Ly, x = random_case(40 + nx, 6, nx, land=0.15, lo=2.0, hi=30.0)
    for adjoint in (False, True):
        g = gpu(mask, Lx, Ly, x, order, K, adjoint)
        o = oracle(mask, Lx, Ly, x, order, K, adjoint)
        assert rel_err(g, o) <= TOL, adjoint


@pytest.mark.parametrize("order,K", FILTERS)
def test_dot_product(regional, order, K):
    mask, Lx, Ly, x = regional
    rng = np.random.default_rng(5)
    y = rng.standard_normal(x.shape).astype(np.float32)
    Vx = gpu(mask, Lx, Ly, x, order, K).astype(np.float64)
    VTy = gpu(mask, Lx, Ly, y, order, K, adjoint=True).astype(np.float64)
    lhs, rhs = np.vdot(Vx, y), np.vdot(x.astype(np.float64), VTy)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Vx) * np.linalg.norm(y)


def test_per_level_masks_and_q_correction():
    """Masks and length scales that differ per level (one coefficient level
    per slice group), with the q-corrected coefficients."""
    rng = np.random.default_rng(8)
    ny, nx, nz = 48, 80, 3
    mask = np.stack([np.roll(synth.land_mask(rng, ny, nx, 4.0, 0.3), 5 * k, axis=1)
                     for k in range(nz)])
    L = np.stack([synth.length_field(rng, ny, nx, 8.0, 2.0, 15.0) * (1 + 0.2 * k)
                  for k in range(nz)]).astype(np.float32)
    x = rng.standard_normal((2, nz, ny, nx)).astype(np.float32)
    for adjoint in (False, True):
        g = gpu(mask, L, 0.7 * L, x, 3, 1, adjoint, qcorr=True)
        o = oracle(mask, L, 0.7 * L, x, 3, 1, adjoint, qcorr=True)
        assert rel_err(g, o) <= TOL


def test_no_imaginary_points_equals_zero_coasts(regional):
    mask, Lx, Ly, x = regional
    a = gpu(mask, Lx, Ly, x, 3, 1, img=0.0, coast="constant")
    b = gpu(mask, Lx, Ly, x, 3, 1, img=0.0, coast="zero")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("order,K", FILTERS)
def test_constant_field_keeps_its_gain_up_to_the_coast(order, K):
    """With 20 sigma of imaginary points a constant field maps to
    2 pi sigma_x sigma_y at every sea point, coastal ones included (uniform
    sigma, Gaussian-peak normalisation), to FP32 accuracy."""
    sigma = 3.0
    rng = np.random.default_rng(12)
    ny, nx = 96, 160
    mask = synth.land_mask(rng, ny, nx, 6.0, 0.3)
    L = np.full((ny, nx), sigma, np.float32)
    x = np.ones((1, 1, ny, nx), np.float32)
    g = gpu(mask, L, L, x, order, K, img=20.0)[0, 0]
    sea = mask == 1
    np.testing.assert_allclose(g[sea], 2 * np.pi * sigma * sigma, rtol=2e-5)
    assert np.all(g[~sea] == 0)


def test_multi_domain_batch_matches_oracle_and_separate_plans():
    doms = synth.ragged_domains(5, scale=0.1, max_levels=12)
    rng = np.random.default_rng(21)
    ny, nx = 10, 1500          # rows on 32 lanes beside the short lines on 16
    doms.append(dict(nx=nx, ny=ny, nz=2, mask=synth.land_mask(rng, ny, nx, 6.0, 0.2),
                     Lx=rng.uniform(2, 30, (ny, nx)).astype(np.float32),
                     Ly=rng.uniform(2, 30, (ny, nx)).astype(np.float32)))
    ny, nx = 8, 4200           # rows on the long-line kernel
    doms.append(dict(nx=nx, ny=ny, nz=1, mask=synth.land_mask(rng, ny, nx, 6.0, 0.2),
                     Lx=rng.uniform(2, 30, (ny, nx)).astype(np.float32),
                     Ly=rng.uniform(2, 30, (ny, nx)).astype(np.float32)))
    xs = [rng.standard_normal((2, d["nz"], d["ny"], d["nx"])).astype(np.float32) for d in doms]
    specs = [dict(mask=d["mask"], Lx=d["Lx"], Ly=d["Ly"], nz=d["nz"]) for d in doms]
    ts = [torch.from_numpy(x).cuda() for x in xs]
    for order, K in FILTERS:
        plan = Plan(specs, opts(order, K))
        fwd, adj = plan.apply(ts), plan.apply_adjoint(ts)
        torch.cuda.synchronize()
        assert plan.status() == 0
        for d, x, f, a in zip(doms, xs, fwd, adj):
            for adjoint, y in ((False, f), (True, a)):
                o = oracle(d["mask"], d["Lx"], d["Ly"], x, order, K, adjoint)
                assert rel_err(y.cpu().numpy(), o) <= TOL, (d["nx"], d["ny"], adjoint)
        for sp, t, f, a in zip(specs, ts, fwd, adj):
            single = Plan(sp, opts(order, K))
            assert torch.equal(single.apply(t), f)
            assert torch.equal(single.apply_adjoint(t), a)
        # tuned shapes (from the constant-extension list) change nothing
        plan.tune(2)
        for t, f in zip(plan.apply(ts), fwd):
            assert torch.equal(t, f)
        text = plan.describe()
        assert "coasts constant extension" in text
        assert "multi-domain" in text or "per-domain" in text


def test_allocation_free_entry_point(regional):
    mask, Lx, Ly, x = regional
    plan = Plan(dict(mask=mask, Lx=Lx, Ly=Ly, nz=x.shape[1]), opts(3, 1))
    xt = torch.from_numpy(x).cuda()
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for adjoint in (False, True):
        out = torch.full_like(xt, float("nan"))
        rc = lib.rf_apply_static(plan.handle, _lib.ptr_array([xt.data_ptr()]),
                                 _lib.ptr_array([out.data_ptr()]), x.shape[0], int(adjoint), stream)
        assert rc == _lib.RF_OK
        torch.cuda.synchronize()
        o = oracle(mask, Lx, Ly, x, 3, 1, adjoint)
        assert rel_err(out.cpu().numpy(), o) <= TOL
