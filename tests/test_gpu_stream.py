"""The streaming column kernel (third-order y pass on coefficients shared by
all levels, zero-input coasts, at least 16384 columns x levels): parity with
the FP64 oracle at the capacity of its segment-end records (13 ends per
column, held in shared memory), the tile kernel taking over at 14 ends and
below 16384 columns x levels, and ragged launch shapes: a column count that
is not a multiple of 32, an odd slice count that leaves half a slice pair,
and slice pairs that fill only part of a CTA's four warps.  Every case runs
forward and adjoint, with imaginary points (coastal maps) and without."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Options, Plan  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
MAX_ENDS = 13
MIN_WORK = 16384   # columns x levels


def column_mask(rng, ny, nx, ends):
    """Mask whose column c has exactly ends[c] sea segments (each at least
    one point, separated by at least one land point, the last one possibly
    reaching the edge), at random rows, so that the lanes of a warp meet
    their segment ends at different steps."""
    m = np.zeros((ny, nx), np.uint8)
    for c, e in enumerate(ends):
        if e == 0:
            continue
        cuts = np.sort(rng.choice(ny + 1, 2 * e, replace=False))
        for k in range(e):
            m[cuts[2 * k]:cuts[2 * k + 1], c] = 1
    return m


def column_ends(m):
    m = m.astype(bool)
    return (m & ~np.vstack([m[1:], np.zeros((1, m.shape[1]), bool)])).sum(0)


def case(seed, ny, nx, nvar, nz, top):
    rng = np.random.default_rng(seed)
    ends = rng.integers(0, top + 1, nx)
    ends[:3] = top          # the capacity itself, on several lanes
    ends[3] = 0             # an all-land column
    m = column_mask(rng, ny, nx, ends)
    m[:, 4] = 1             # an all-sea column: one end, at the edge
    assert column_ends(m).max() == top
    L = rng.uniform(1.0, 12.0, (ny, nx)).astype(np.float32)
    Ly = rng.uniform(1.0, 12.0, (ny, nx)).astype(np.float32)
    x = rng.standard_normal((nvar, nz, ny, nx)).astype(np.float32)
    return m, L, Ly, x


def run(m, L, Ly, x, adjoint, img):
    plan = Plan(dict(mask=m, Lx=L, Ly=Ly, nz=x.shape[1]), Options(order=3, iters=1, img_factor=img))
    xt = torch.from_numpy(x).cuda()
    y = plan.apply_adjoint(xt) if adjoint else plan.apply(xt)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return y.cpu().numpy(), plan.describe()


def oracle(m, L, Ly, x, adjoint, img):
    return orc.vh(x.astype(np.float64), m, L.astype(np.float64), Ly.astype(np.float64),
                  order=3, iters=1, adjoint=adjoint, img_factor=img)


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("top,nz,streams", [(MAX_ENDS, 16, True), (MAX_ENDS + 1, 16, False),
                                            (MAX_ENDS, 15, False)])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("img", [3.0, 0.0])
def test_record_capacity(top, nz, streams, adjoint, img):
    nx = 1030
    assert (nx * nz >= MIN_WORK) == (nz == 16)
    m, L, Ly, x = case(11 + top, 120, nx, 1, nz, top)
    y, text = run(m, L, Ly, x, adjoint, img)
    assert ("streaming column kernel" in text) == streams, text
    ref = oracle(m, L, Ly, x, adjoint, img)
    assert rel_err(y, ref) <= TOL
    assert np.all(y[:, :, m == 0] == 0)


@pytest.mark.parametrize("nvar,nz,nx", [(1, 1, 16400), (2, 5, 3300), (2, 9, 1850)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_ragged_launch_shapes(nvar, nz, nx, adjoint):
    assert nx % 32 and nx * nz >= MIN_WORK
    m, L, Ly, x = case(5 + nz, 97, nx, nvar, nz, 9)
    y, text = run(m, L, Ly, x, adjoint, 3.0)
    assert "streaming column kernel" in text, text
    ref = oracle(m, L, Ly, x, adjoint, 3.0)
    for v in range(nvar):
        for k in range(nz):
            assert rel_err(y[v, k], ref[v, k]) <= TOL, (v, k)
