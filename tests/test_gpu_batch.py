"""Ragged multi-domain batches: one persistent launch per pass over a work
list of the tile-kernel domains' (line block, slice group) items (domains on
the register kernel launch on their own), and CUDA graphs of a whole
application.  Parity with the FP64 oracle per domain (bar 1e-5 of the
domain's max |oracle|); the multi-domain launch, separate per-domain plans,
tuned shapes and graph replays must agree bit for bit, since none of them
changes the arithmetic of a slice."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Options, Plan, synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
FILTERS = [(3, 1), (1, 5)]
NVAR = 2


def batch():
    """Small ragged domains (seeded recipe of the 64-domain batch, shrunk),
    one domain whose rows are too long for the tile kernel (4200 points), one
    whose rows (1500 points) run with 32 lanes per line where the short lines
    of the 3rd-RF run with 16, and one with a mask and length scales that
    differ per level."""
    doms = synth.ragged_domains(6, scale=0.1, max_levels=20)
    rng = np.random.default_rng(55)
    ny, nx = 8, 1500
    L = (3.0 + 30.0 * rng.random((ny, nx))).astype(np.float32)
    m = synth.land_mask(rng, ny, nx, 6.0, 0.2)
    doms.append(dict(nx=nx, ny=ny, nz=2, mask=m, Lx=L, Ly=L.copy()))
    ny, nx = 12, 4200
    L = (3.0 + 20.0 * rng.random((ny, nx))).astype(np.float32)
    m = (rng.random((ny, nx)) > 0.1).astype(np.uint8)
    doms.append(dict(nx=nx, ny=ny, nz=2, mask=m, Lx=L, Ly=L.copy()))
    ny, nx, nz = 40, 70, 3
    m3 = np.stack([np.roll(synth.land_mask(rng, ny, nx, 4.0, 0.3), 3 * k, axis=1) for k in range(nz)])
    L3 = np.stack([synth.length_field(rng, ny, nx, 8.0, 3.0, 12.0) * (1 + 0.2 * k) for k in range(nz)])
    doms.append(dict(nx=nx, ny=ny, nz=nz, mask=m3, Lx=L3.astype(np.float32),
                     Ly=(0.8 * L3).astype(np.float32)))
    xs = [rng.standard_normal((NVAR, d["nz"], d["ny"], d["nx"])).astype(np.float32) for d in doms]
    return doms, xs


def reg_shape(m):
    """(chunk length, lanes per line) of the register kernel for lines of m
    points: the first built shape that covers the line."""
    for C, P in [(16, 8), (16, 16), (24, 16), (16, 32), (24, 32), (32, 32)]:
        if C * P >= m:
            return C, P


STREAM_MAX_ENDS = 13   # segment ends per column the streaming kernel's records hold
STREAM_MIN_WORK = 16384   # columns x levels of a domain below which the tile kernel serves


def column_ends(mask):
    """Most segment ends (a sea point followed by land or the edge) on one
    column of a 2-D mask."""
    m = np.asarray(mask).astype(bool)
    return int((m & ~np.vstack([m[1:], np.zeros((1, m.shape[1]), bool)])).sum(0).max())


def expected_launches(doms, order):
    """Kernel launches of one application of the batch: per pass, one
    multi-domain register-kernel launch per chunk shape of the domains whose
    lines (at most 1024 points, coefficients shared by all levels; for the
    3rd-RF the rows only) run on the register kernel, one multi-domain launch
    of the streaming column kernel for the third-order columns of domains
    with shared coefficients, at most STREAM_MAX_ENDS segment ends per
    column and at least STREAM_MIN_WORK columns x levels, one for every domain on the long-line kernel (lines over 4064
    points), and one multi-domain launch per lanes-per-line group of the
    remaining tile-kernel domains (16 lanes for third-order lines of at most
    512 points, else 32)."""
    n = 0
    for along_x in (True, False):
        groups, shapes, streams = set(), set(), 0
        for d in doms:
            shared = np.asarray(d["mask"]).ndim == 2 and np.asarray(d["Lx"]).ndim == 2
            m = d["nx"] if along_x else d["ny"]
            if shared and m <= 1024 and (along_x or order == 1):
                shapes.add(reg_shape(m))
            elif (shared and not along_x and order == 3
                  and column_ends(d["mask"]) <= STREAM_MAX_ENDS
                  and d["nx"] * d["nz"] >= STREAM_MIN_WORK):
                streams = 1   # the streaming column kernel, one launch for all
            elif m > 4064:
                n += 1
            else:
                groups.add(16 if order == 3 and m <= 512 else 32)
        n += len(groups) + len(shapes) + streams
    return n


def plan_of(doms, order, K):
    return Plan([dict(mask=d["mask"], Lx=d["Lx"], Ly=d["Ly"], nz=d["nz"]) for d in doms],
                Options(order=order, iters=K))


def oracle_of(d, x, order, K, adjoint):
    return orc.vh(x.astype(np.float64), d["mask"], np.asarray(d["Lx"], np.float64),
                  np.asarray(d["Ly"], np.float64), order=order, iters=K, adjoint=adjoint)


@pytest.fixture(scope="module")
def data():
    return batch()


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_ragged_batch_matches_oracle(data, order, K, adjoint):
    doms, xs = data
    plan = plan_of(doms, order, K)
    ts = [torch.from_numpy(x).cuda() for x in xs]
    ys = plan.apply_adjoint(ts) if adjoint else plan.apply(ts)
    torch.cuda.synchronize()
    assert plan.status() == 0
    for d, x, y in zip(doms, xs, ys):
        o = oracle_of(d, x, order, K, adjoint)
        err = np.abs(y.cpu().numpy() - o).max() / max(np.abs(o).max(), 1e-300)
        assert err <= TOL, (d["nx"], d["ny"], d["nz"], err)


@pytest.mark.parametrize("order,K", FILTERS)
def test_multi_domain_launch_equals_separate_plans(data, order, K):
    doms, xs = data
    plan = plan_of(doms, order, K)
    ts = [torch.from_numpy(x).cuda() for x in xs]
    launches0 = plan.info()[3]
    fwd, adj = plan.apply(ts), plan.apply_adjoint(ts)
    assert plan.info()[3] - launches0 == 2 * expected_launches(doms, order)
    text = plan.describe()
    for dirname in ("x", "y"):
        assert f"multi-domain {dirname} forward" in text
    for d, t, f, a in zip(doms, ts, fwd, adj):
        single = plan_of([d], order, K)
        assert torch.equal(single.apply(t), f)
        assert torch.equal(single.apply_adjoint(t), a)


def test_tuned_batch_gives_identical_results(data):
    doms, xs = data
    ts = [torch.from_numpy(x).cuda() for x in xs]
    for order, K in FILTERS:
        plan = plan_of(doms, order, K)
        ref_f, ref_a = plan.apply(ts), plan.apply_adjoint(ts)
        plan.tune(NVAR)
        for a, b in zip(plan.apply(ts), ref_f):
            assert torch.equal(a, b)
        for a, b in zip(plan.apply_adjoint(ts), ref_a):
            assert torch.equal(a, b)
        assert plan.status() == 0


@pytest.mark.parametrize("adjoint", [False, True])
def test_graph_replays_the_application(data, adjoint):
    doms, xs = data
    plan = plan_of(doms, 3, 1)
    ts = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.empty_like(t) for t in ts]
    g = plan.graph(ts, outs, adjoint=adjoint)
    rng = np.random.default_rng(9)
    for _ in range(2):   # new input contents each replay
        for t in ts:
            t.copy_(torch.from_numpy(rng.standard_normal(tuple(t.shape)).astype(np.float32)))
        launches0 = plan.info()[3]
        g.launch()
        torch.cuda.synchronize()
        assert plan.info()[3] > launches0
        ref = plan.apply_adjoint(ts) if adjoint else plan.apply(ts)
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)
    g.close()
    assert plan.status() == 0


def test_graph_of_a_single_domain_plan():
    w = synth.workload(2, nz=3, nvar=NVAR)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=3))
    x = torch.from_numpy(w["x"]).cuda()
    y = torch.empty_like(x)
    g = plan.graph(x, y)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(y, plan.apply(x))
    g.close()
