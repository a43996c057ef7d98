"""Carried coasts (RF_FLAG_COAST_CARRIED, 1st-RF x K): the imaginary sea
points start at zero and keep their values from one iteration to the next
(each segment is extended once, filtered K times, read back once), another
of the coastal conditions the paper's Conclusions leave for future work.
Parity with the FP64 oracle's carried coasts (bar 1e-5 of max |oracle|)
through the register kernel (lines of up to 1024 points), the long-line
kernel (longer lines, per-level masks) and the allocation-free entry point;
finite and infinite imaginary seas; the GPU dot test; K = 1 and the 3rd-RF
reduce to zero-input coasts bit for bit."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Options, Plan, _lib, synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def opts(K, img=3.0, coast="carried", order=1):
    return Options(order=order, iters=K, img_factor=img, coast=coast)


def plan_of(mask, Lx, Ly, nz, K, img=3.0, coast="carried", order=1):
    return Plan(dict(mask=mask, Lx=Lx, Ly=Ly, nz=nz), opts(K, img, coast, order))


def gpu(mask, Lx, Ly, x, K, adjoint=False, img=3.0, coast="carried", order=1):
    plan = plan_of(mask, Lx, Ly, x.shape[1], K, img, coast, order)
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    y = plan.apply_adjoint(xt) if adjoint else plan.apply(xt)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return y.cpu().numpy()


def oracle(mask, Lx, Ly, x, K, adjoint=False, img=3.0):
    return orc.vh(np.asarray(x, np.float64), mask, np.asarray(Lx, np.float64),
                  np.asarray(Ly, np.float64), order=1, iters=K, adjoint=adjoint,
                  img_factor=img, coast=orc.COAST_CARRIED)


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


@pytest.mark.parametrize("K", [2, 5])
@pytest.mark.parametrize("adjoint", [False, True])
def test_regional_grid_matches_oracle(regional, K, adjoint):
    """1024 x 384 with coastlines: the register kernel (rows on 32 lanes,
    columns on 16)."""
    mask, Lx, Ly, x = regional
    plan = plan_of(mask, Lx, Ly, x.shape[1], K)
    text = plan.describe()
    assert "carried across iterations" in text and "register kernel" in text
    g = gpu(mask, Lx, Ly, x, K, adjoint)
    o = oracle(mask, Lx, Ly, x, K, adjoint)
    assert rel_err(g, o) <= TOL
    # the option changes the result near the coasts
    z = gpu(mask, Lx, Ly, x, K, adjoint, coast="zero")
    assert rel_err(z, o) > 1e-4


@pytest.mark.parametrize("adjoint", [False, True])
def test_infinite_imaginary_sea(regional, adjoint):
    mask, Lx, Ly, x = regional
    g = gpu(mask, Lx, Ly, x, 5, adjoint, img=np.inf)
    o = oracle(mask, Lx, Ly, x, 5, adjoint, img=np.inf)
    assert rel_err(g, o) <= TOL


EDGE_GRIDS = [(1, 1), (1, 7), (9, 1), (3, 5), (17, 13), (33, 65), (130, 3)]


@pytest.mark.parametrize("ny,nx", EDGE_GRIDS)
def test_small_and_ragged_grids(ny, nx):
    """Grid-edge segment starts, one-point segments and chunks past the
    line's end."""
    mask, Lx, Ly, x = random_case(ny * 100 + nx, ny, nx, land=0.3, lo=0.5)
    for adjoint in (False, True):
        g = gpu(mask, Lx, Ly, x, 5, adjoint)
        o = oracle(mask, Lx, Ly, x, 5, adjoint)
        if np.abs(o).max() == 0:
            assert np.all(g == 0)
        else:
            assert rel_err(g, o) <= TOL, adjoint


@pytest.mark.parametrize("nx", [300, 1000, 1500, 4200])
def test_line_lengths_across_kernels(nx):
    """Rows of 300 and 1000 points (register kernel), 1500 and 4200 (the
    long-line kernel)."""
    mask, Lx, Ly, x = random_case(60 + nx, 6, nx, land=0.15, lo=2.0, hi=30.0)
    for adjoint in (False, True):
        g = gpu(mask, Lx, Ly, x, 5, adjoint)
        o = oracle(mask, Lx, Ly, x, 5, adjoint)
        assert rel_err(g, o) <= TOL, adjoint


def test_per_level_masks():
    """Masks and length scales that differ per level (the long-line kernel)."""
    rng = np.random.default_rng(18)
    ny, nx, nz = 48, 80, 3
    mask = np.stack([np.roll(synth.land_mask(rng, ny, nx, 4.0, 0.3), 5 * k, axis=1)
                     for k in range(nz)])
    L = np.stack([synth.length_field(rng, ny, nx, 8.0, 2.0, 15.0) * (1 + 0.2 * k)
                  for k in range(nz)]).astype(np.float32)
    x = rng.standard_normal((2, nz, ny, nx)).astype(np.float32)
    for adjoint in (False, True):
        g = gpu(mask, L, 0.7 * L, x, 4, adjoint)
        o = oracle(mask, L, 0.7 * L, x, 4, adjoint)
        assert rel_err(g, o) <= TOL


def test_dot_product(regional):
    mask, Lx, Ly, x = regional
    rng = np.random.default_rng(9)
    y = rng.standard_normal(x.shape).astype(np.float32)
    Vx = gpu(mask, Lx, Ly, x, 5).astype(np.float64)
    VTy = gpu(mask, Lx, Ly, y, 5, adjoint=True).astype(np.float64)
    lhs, rhs = np.vdot(Vx, y), np.vdot(x.astype(np.float64), VTy)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Vx) * np.linalg.norm(y)


def test_reductions_to_zero_coasts(regional):
    """One iteration, the 3rd-RF and no imaginary points: carried coasts are
    the zero-input coasts, bit for bit."""
    mask, Lx, Ly, x = regional
    for order, K, img in [(1, 1, 3.0), (3, 1, 3.0), (1, 5, 0.0)]:
        for adjoint in (False, True):
            a = gpu(mask, Lx, Ly, x, K, adjoint, img=img, order=order)
            b = gpu(mask, Lx, Ly, x, K, adjoint, img=img, order=order, coast="zero")
            assert np.array_equal(a, b), (order, K, img, adjoint)


def test_allocation_free_entry_point(regional):
    mask, Lx, Ly, x = regional
    plan = plan_of(mask, Lx, Ly, x.shape[1], 5)
    xt = torch.from_numpy(x).cuda()
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for adjoint in (False, True):
        out = torch.full_like(xt, float("nan"))
        rc = lib.rf_apply_static(plan.handle, _lib.ptr_array([xt.data_ptr()]),
                                 _lib.ptr_array([out.data_ptr()]), x.shape[0], int(adjoint), stream)
        assert rc == _lib.RF_OK
        torch.cuda.synchronize()
        o = oracle(mask, Lx, Ly, x, 5, adjoint)
        assert rel_err(out.cpu().numpy(), o) <= TOL
