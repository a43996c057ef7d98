"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: max |gpu - oracle| <= 1e-5 * max |oracle| per field (FP32 recursion
against the FP64 oracle), the adjoint dot test <Vx,y> - <x,V^T y> within
1e-5 of ||Vx|| ||y|| in FP32.  Inputs come from the seeded generators.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Options, Plan, synth, vh  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5

FILTERS = [(3, 1), (1, 5)]


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def run_gpu(w, x, order, K, adjoint=False, img=3.0, norm=0, mask=None, Lx=None, Ly=None):
    mask = w["mask"] if mask is None else mask
    Lx = w["Lx"] if Lx is None else Lx
    Ly = w["Ly"] if Ly is None else Ly
    plan = Plan(dict(mask=mask, Lx=Lx, Ly=Ly, nz=x.shape[1]),
                Options(order=order, iters=K, img_factor=img, norm=norm))
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = plan.apply_adjoint(xt) if adjoint else plan.apply(xt)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return y.cpu().numpy()


def run_oracle(w, x, order, K, adjoint=False, img=3.0, norm=0, mask=None, Lx=None, Ly=None):
    mask = w["mask"] if mask is None else mask
    Lx = w["Lx"] if Lx is None else Lx
    Ly = w["Ly"] if Ly is None else Ly
    return orc.vh(x.astype(np.float64), mask, np.asarray(Lx, np.float64),
                  np.asarray(Ly, np.float64), order=order, iters=K,
                  adjoint=adjoint, img_factor=img, norm=norm)


@pytest.fixture(scope="module")
def cfg1():
    return synth.workload(1)


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_impulse_256x128(cfg1, order, K, adjoint):
    x = synth.impulse(128, 256, 64, 128)
    g = run_gpu(cfg1, x, order, K, adjoint)
    o = run_oracle(cfg1, x, order, K, adjoint)
    assert rel_err(g, o) <= TOL


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_noise_256x128(cfg1, order, K, adjoint):
    x = cfg1["x"]
    g = run_gpu(cfg1, x, order, K, adjoint)
    o = run_oracle(cfg1, x, order, K, adjoint)
    assert rel_err(g, o) <= TOL


@pytest.fixture(scope="module")
def cfg2_small():
    return synth.workload(2, nz=2, nvar=2)


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_regional_1024x384_with_coasts(cfg2_small, order, K, adjoint):
    w = cfg2_small
    g = run_gpu(w, w["x"], order, K, adjoint)
    o = run_oracle(w, w["x"], order, K, adjoint)
    for v in range(w["nvar"]):
        for k in range(w["nz"]):
            assert rel_err(g[v, k], o[v, k]) <= TOL
    assert np.all(g[:, :, w["mask"] == 0] == 0.0)


@pytest.mark.parametrize("adjoint", [False, True])
def test_global_1440x1080_latitude_scales(adjoint):
    w = synth.workload(3, nz=1)
    g = run_gpu(w, w["x"], 3, 1, adjoint)
    o = run_oracle(w, w["x"], 3, 1, adjoint)
    assert rel_err(g, o) <= TOL


@pytest.mark.parametrize("order,K", FILTERS)
def test_gpu_dot_product(cfg2_small, order, K):
    w = cfg2_small
    rng = np.random.default_rng(4)
    y = rng.standard_normal(w["x"].shape).astype(np.float32)
    Vx = run_gpu(w, w["x"], order, K).astype(np.float64)
    VTy = run_gpu(w, y, order, K, adjoint=True).astype(np.float64)
    lhs, rhs = np.vdot(Vx, y), np.vdot(w["x"].astype(np.float64), VTy)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Vx) * np.linalg.norm(y)


# ------------------------------------------------------------ edge cases
EDGE_GRIDS = [(1, 1), (1, 7), (9, 1), (3, 5), (17, 13), (33, 65), (130, 3)]


@pytest.mark.parametrize("ny,nx", EDGE_GRIDS)
@pytest.mark.parametrize("order,K", [(3, 1), (1, 5), (1, 1)])
def test_small_and_ragged_grids(ny, nx, order, K):
    rng = np.random.default_rng(ny * 1000 + nx)
    mask = (rng.uniform(size=(ny, nx)) > 0.3).astype(np.uint8)
    L = rng.uniform(0.5, 12.0, (ny, nx)).astype(np.float32)
    Ly = rng.uniform(0.5, 12.0, (ny, nx)).astype(np.float32)
    w = dict(mask=mask, Lx=L, Ly=Ly)
    x = rng.standard_normal((2, 3, ny, nx)).astype(np.float32)
    for adjoint in (False, True):
        g = run_gpu(w, x, order, K, adjoint)
        o = run_oracle(w, x, order, K, adjoint)
        if np.abs(o).max() == 0:
            assert np.all(g == 0)
        else:
            assert rel_err(g, o) <= TOL


@pytest.mark.parametrize("img,norm", [(0.0, 0), (1.0, 1), (7.5, 0)])
def test_options_img_factor_and_norm(cfg2_small, img, norm):
    w = cfg2_small
    x = w["x"][:, :1]
    for order, K in FILTERS:
        g = run_gpu(w, x, order, K, img=img, norm=norm)
        o = run_oracle(w, x, order, K, img=img, norm=norm)
        assert rel_err(g, o) <= TOL


@pytest.mark.parametrize("adjoint", [False, True])
def test_infinite_imaginary_sea(cfg2_small, adjoint):
    """img_factor = inf: the plan's closed-form limit map (the Stein equation
    of the boundary map, FP64) against the oracle's explicit extension cut
    below FP64 resolution, on the coastal regional grid (length scales up to
    40), both filters; and the limit is approached by a long finite sea."""
    w = cfg2_small
    x = w["x"][:, :1]
    for order, K in FILTERS:
        g = run_gpu(w, x, order, K, adjoint, img=float("inf"))
        o = run_oracle(w, x, order, K, adjoint, img=float("inf"))
        assert rel_err(g, o) <= TOL
        far = run_gpu(w, x, order, K, adjoint, img=60.0)
        assert rel_err(far, g) <= TOL


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("img,norm", [(3.0, 0), (0.0, 1)])
def test_q_corrected_filter(cfg2_small, cfg1, adjoint, img, norm):
    """The q-corrected 3rd-RF (an option, not the paper's filter) against the
    oracle's, on the coastal regional grid and the impulse grid."""
    for w in (cfg2_small, cfg1):
        x = np.ascontiguousarray(w["x"][:, :1])
        plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=1),
                    Options(img_factor=img, norm=norm, qcorr=True))
        xt = torch.from_numpy(x).cuda()
        g = (plan.apply_adjoint(xt) if adjoint else plan.apply(xt)).cpu().numpy()
        o = orc.vh(x.astype(np.float64), w["mask"], np.asarray(w["Lx"], np.float64),
                   np.asarray(w["Ly"], np.float64), adjoint=adjoint, img_factor=img,
                   norm=norm, qcorr=True)
        assert rel_err(g, o) <= TOL
        assert plan.status() == 0


def test_q_correction_needs_the_third_order_filter(cfg1):
    w = cfg1
    with pytest.raises(Exception):
        Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=1),
             Options(order=1, iters=5, qcorr=True))


def test_all_land_and_all_sea():
    ny, nx = 20, 24
    L = np.full((ny, nx), 3.0, np.float32)
    x = np.random.default_rng(0).standard_normal((1, 1, ny, nx)).astype(np.float32)
    land = dict(mask=np.zeros((ny, nx), np.uint8), Lx=L, Ly=L)
    assert np.all(run_gpu(land, x, 3, 1) == 0)
    sea = dict(mask=np.ones((ny, nx), np.uint8), Lx=L, Ly=L)
    assert rel_err(run_gpu(sea, x, 3, 1), run_oracle(sea, x, 3, 1)) <= TOL


def test_level_dependent_mask_and_length_scales():
    rng = np.random.default_rng(8)
    nz, ny, nx = 4, 40, 50
    mask = (rng.uniform(size=(nz, ny, nx)) > 0.2).astype(np.uint8)
    Lx = rng.uniform(1.0, 15.0, (nz, ny, nx)).astype(np.float32)
    Ly = rng.uniform(1.0, 15.0, (nz, ny, nx)).astype(np.float32)
    w = dict(mask=mask, Lx=Lx, Ly=Ly)
    x = rng.standard_normal((2, nz, ny, nx)).astype(np.float32)
    for order, K in FILTERS:
        for adjoint in (False, True):
            assert rel_err(run_gpu(w, x, order, K, adjoint),
                           run_oracle(w, x, order, K, adjoint)) <= TOL


def test_large_length_scale_fp32_accuracy():
    """sigma = 40 on 1024-point lines: the delta realisation keeps FP32 error
    far below the bound where the direct form would not."""
    ny, nx = 64, 1024
    L = np.full((ny, nx), 40.0, np.float32)
    w = dict(mask=np.ones((ny, nx), np.uint8), Lx=L, Ly=L)
    x = np.random.default_rng(1).standard_normal((1, 1, ny, nx)).astype(np.float32)
    for adjoint in (False, True):
        assert rel_err(run_gpu(w, x, 3, 1, adjoint), run_oracle(w, x, 3, 1, adjoint)) <= 2e-6


def test_in_place_and_multi_domain():
    rng = np.random.default_rng(12)
    doms = synth.ragged_domains(5, scale=0.12, max_levels=3)
    opts = Options()
    plan = Plan([dict(mask=d["mask"], Lx=d["Lx"], Ly=d["Ly"], nz=d["nz"]) for d in doms], opts)
    xs = [rng.standard_normal((2, d["nz"], d["ny"], d["nx"])).astype(np.float32) for d in doms]
    ts = [torch.from_numpy(x).cuda() for x in xs]
    outs = plan.apply(ts, out=ts)          # in place
    torch.cuda.synchronize()
    for d, x, y in zip(doms, xs, outs):
        o = run_oracle(d, x, 3, 1)
        assert rel_err(y.cpu().numpy(), o) <= TOL


def test_apply_host_matches_device():
    w = synth.workload(1)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=1))
    x = torch.from_numpy(w["x"]).contiguous()
    out = torch.empty_like(x).pin_memory()
    plan.apply_host(x.pin_memory(), out, nvar=1)
    ref = plan.apply(x.cuda()).cpu()
    assert torch.equal(out, ref)
    plan.apply_host(x.pin_memory(), out, nvar=1, adjoint=True)
    assert torch.equal(out, plan.apply_adjoint(x.cuda()).cpu())


@pytest.mark.parametrize("order,K", FILTERS)
def test_apply_host_pipeline_over_level_batches(order, K):
    """20 levels go through the host-buffer call in 7 level batches whose
    copies and launches overlap; a second, ragged domain shares the plan.
    The result must equal the device call bit for bit, also in place."""
    w = synth.workload(2, nz=20, nvar=2)
    doms = [dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=20)]
    d2 = synth.ragged_domains(1, scale=0.15, max_levels=40)[0]
    doms.append(dict(mask=d2["mask"], Lx=d2["Lx"], Ly=d2["Ly"], nz=d2["nz"]))
    plan = Plan(doms, Options(order=order, iters=K))
    rng = np.random.default_rng(21)
    xs = [torch.from_numpy(w["x"]),
          torch.from_numpy(rng.standard_normal((2, d2["nz"], d2["ny"], d2["nx"])).astype(np.float32))]
    xs = [x.contiguous().pin_memory() for x in xs]
    for adjoint in (False, True):
        outs = [torch.empty_like(x).pin_memory() for x in xs]
        plan.apply_host(xs, outs, nvar=2, adjoint=adjoint)
        dev = [x.cuda() for x in xs]
        ref = plan.apply_adjoint(dev) if adjoint else plan.apply(dev)
        for o, r in zip(outs, ref):
            assert torch.equal(o, r.cpu())
        inplace = [x.clone().pin_memory() for x in xs]
        plan.apply_host(inplace, inplace, nvar=2, adjoint=adjoint)
        for o, r in zip(inplace, ref):
            assert torch.equal(o, r.cpu())
    assert plan.status() == 0


def test_autograd_backward_is_adjoint_and_matches_finite_differences():
    """J(v) = 1/2 ||H V v - y||^2 with H a sampling of sea points: the autograd
    gradient equals V^T H^T (H V v - y) and a central difference (exact up to
    rounding for a quadratic J)."""
    w = synth.workload(2, nz=2, nvar=2)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=2))
    rng = np.random.default_rng(44)
    sea = np.flatnonzero(np.broadcast_to(w["mask"], (2, 2) + w["mask"].shape).ravel())
    idx = torch.from_numpy(rng.choice(sea, 5000, replace=False)).cuda()
    yobs = torch.from_numpy(rng.normal(0, 0.5, 5000).astype(np.float32)).cuda()
    v = torch.from_numpy(w["x"]).cuda().requires_grad_(True)

    def J(vv):
        r = vh(vv, plan).reshape(-1)[idx] - yobs
        return 0.5 * (r * r).sum()

    j = J(v)
    j.backward()
    r = (plan.apply(v.detach()).reshape(-1)[idx] - yobs)
    ht = torch.zeros(v.numel(), device="cuda").index_add_(0, idx, r).reshape(v.shape)
    ref = plan.apply_adjoint(ht)
    assert torch.allclose(v.grad, ref, rtol=0, atol=1e-6 * ref.abs().max().item())
    d = torch.from_numpy(rng.standard_normal(w["x"].shape).astype(np.float32)).cuda()
    with torch.no_grad():
        fd = (J(v + d).double() - J(v - d).double()) / 2.0
    an = (v.grad.double() * d.double()).sum()
    assert abs(fd.item() - an.item()) <= 1e-4 * abs(an.item())


def test_tuned_shapes_give_identical_results():
    """The autotuner only changes launch shapes and level batches, never the
    kernel of a direction or the arithmetic of a slice: results are
    bit-identical."""
    w = synth.workload(2, nz=3, nvar=2)
    x = torch.from_numpy(w["x"]).cuda()
    for order, K in FILTERS:
        plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=3), Options(order=order, iters=K))
        ref_f, ref_a = plan.apply(x), plan.apply_adjoint(x)
        plan.tune(2)
        assert torch.equal(plan.apply(x), ref_f)
        assert torch.equal(plan.apply_adjoint(x), ref_a)
        assert plan.status() == 0
        text = plan.describe()
        assert "x: lines 384 of 1024 points" in text and "register kernel C=32 P=32" in text


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("nx", [3000, 4200])
def test_long_lines(order, K, nx):
    """Rows of 3000 points fill chunks of 95 points, so segment ends fall in
    both halves of the tile kernel's 128-bit per-chunk masks.  Rows of 4200
    points are longer than the tile kernel takes (32 chunks of at most 127
    points): the one-thread-per-line kernel with its global scratch for the
    coastal start states filters them."""
    rng = np.random.default_rng(30)
    ny = 6
    mask = (rng.uniform(size=(ny, nx)) > 0.15).astype(np.uint8)
    L = rng.uniform(2.0, 30.0, (ny, nx)).astype(np.float32)
    w = dict(mask=mask, Lx=L, Ly=L)
    x = rng.standard_normal((2, 2, ny, nx)).astype(np.float32)
    for adjoint in (False, True):
        assert rel_err(run_gpu(w, x, order, K, adjoint), run_oracle(w, x, order, K, adjoint)) <= TOL


@pytest.mark.parametrize("order,K", FILTERS)
def test_lanes_per_line_switch(order, K):
    """Third-order lines of up to 512 points run with 16 lanes per line
    (chunks of 33 points at 512), longer ones with 32 (chunks of 17 at 513);
    the first-order filter always uses 32.  Rows of 513 and columns of 512
    points put both kinds in one application."""
    rng = np.random.default_rng(31)
    ny, nx = 512, 513
    mask = (rng.uniform(size=(ny, nx)) > 0.2).astype(np.uint8)
    L = rng.uniform(2.0, 30.0, (ny, nx)).astype(np.float32)
    Ly = rng.uniform(2.0, 30.0, (ny, nx)).astype(np.float32)
    w = dict(mask=mask, Lx=L, Ly=Ly)
    x = rng.standard_normal((2, 2, ny, nx)).astype(np.float32)
    for adjoint in (False, True):
        assert rel_err(run_gpu(w, x, order, K, adjoint), run_oracle(w, x, order, K, adjoint)) <= TOL
    text = Plan(dict(mask=mask, Lx=L, Ly=Ly, nz=2), Options(order=order, iters=K)).describe()
    assert "x: lines 512 of 513 points, 32 lanes per line, chunk 17" in text
    lanes_y = "16 lanes per line, chunk 33" if order == 3 else "32 lanes per line, chunk 17"
    assert f"y: lines 513 of 512 points, {lanes_y}" in text
