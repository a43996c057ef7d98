"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: the regional basin 1024 x 384 x 72 with T and S after
autotuning, the global grid 1440 x 1080 x 75, and the 64-domain ragged batch
through CUDA graphs of tuned multi-domain launches.  The oracle computes
sampled level slices one by one (bar 1e-5 of max |oracle| per slice); the
whole-field dot test holds at any size (1e-5 of ||Vx|| ||y||, FP64 sums of
the FP32 results)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Options, Plan, synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def slice_oracle(mask, Lx, Ly, s, adjoint=False):
    return orc.vh(np.asarray(s, np.float64), mask, np.asarray(Lx, np.float64),
                  np.asarray(Ly, np.float64), adjoint=adjoint)


def dot_residual(x, Vx, VTy, y):
    lhs = float((Vx.double() * y.double()).sum())
    rhs = float((x.double() * VTy.double()).sum())
    return abs(lhs - rhs) / (float(Vx.double().norm()) * float(y.double().norm()))


@pytest.fixture(scope="module")
def regional():
    w = synth.workload(2)
    assert (w["nz"], w["ny"], w["nx"], w["nvar"]) == (72, 384, 1024, 2)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=w["nz"]), Options(order=3))
    plan.tune(w["nvar"])
    return w, plan


def test_regional_full_size_tuned(regional):
    w, plan = regional
    x = torch.from_numpy(w["x"]).cuda()
    y = plan.apply(x)
    z = plan.apply_adjoint(x)
    torch.cuda.synchronize()
    assert plan.status() == 0
    for v, k in [(0, 0), (0, 37), (1, 71)]:
        s = w["x"][v, k]
        assert rel_err(y[v, k].cpu().numpy(), slice_oracle(w["mask"], w["Lx"], w["Ly"], s)) <= TOL
        assert rel_err(z[v, k].cpu().numpy(),
                       slice_oracle(w["mask"], w["Lx"], w["Ly"], s, adjoint=True)) <= TOL
    rng = np.random.default_rng(72)
    u = torch.from_numpy(rng.standard_normal(w["x"].shape).astype(np.float32)).cuda()
    VTu = plan.apply_adjoint(u)
    assert dot_residual(x, y, VTu, u) <= TOL


def test_global_full_size():
    w = synth.workload(3)
    assert (w["nz"], w["ny"], w["nx"]) == (75, 1080, 1440)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=w["nz"]), Options(order=3))
    x = torch.from_numpy(w["x"]).cuda()
    y = plan.apply(x)
    z = plan.apply_adjoint(x)
    torch.cuda.synchronize()
    assert plan.status() == 0
    for k in (0, 74):
        s = w["x"][0, k]
        assert rel_err(y[0, k].cpu().numpy(), slice_oracle(w["mask"], w["Lx"], w["Ly"], s)) <= TOL
        assert rel_err(z[0, k].cpu().numpy(),
                       slice_oracle(w["mask"], w["Lx"], w["Ly"], s, adjoint=True)) <= TOL


def test_ragged_64_domains_tuned_graphs():
    """The benchmark's ragged batch (64 seeded domains, one variable), tuned
    multi-domain launches replayed as CUDA graphs; three domains' first and
    last levels checked against the oracle."""
    doms = synth.ragged_domains(64)
    specs = [dict(mask=d["mask"], Lx=d["Lx"], Ly=d["Ly"], nz=d["nz"]) for d in doms]
    plan = Plan(specs, Options(order=3))
    plan.tune_batch(1)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1405)
    xs = [torch.randn((1, d["nz"], d["ny"], d["nx"]), generator=gen, device="cuda") for d in doms]
    ys = [torch.empty_like(x) for x in xs]
    zs = [torch.empty_like(x) for x in xs]
    g_f = plan.graph(xs, ys)
    g_a = plan.graph(xs, zs, adjoint=True)
    g_f.launch()
    g_a.launch()
    torch.cuda.synchronize()
    assert plan.status() == 0
    sizes = [d["nx"] * d["ny"] for d in doms]
    picks = [int(np.argmax(sizes)), int(np.argmin(sizes)), 17]
    for i in picks:
        d = doms[i]
        for k in sorted({0, d["nz"] - 1}):
            s = xs[i][0, k].cpu().numpy()
            assert rel_err(ys[i][0, k].cpu().numpy(), slice_oracle(d["mask"], d["Lx"], d["Ly"], s)) <= TOL
            assert rel_err(zs[i][0, k].cpu().numpy(),
                           slice_oracle(d["mask"], d["Lx"], d["Ly"], s, adjoint=True)) <= TOL
    g_f.close()
    g_a.close()
