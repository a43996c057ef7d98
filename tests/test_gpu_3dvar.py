"""V_H inside the 3D-VAR cost it serves (Eq. "eight"): J(v) = 1/2 ||H V_H v - y||^2
with H bilinear interpolation at 50,000 observations on the regional grid
(4 levels, T and S), observation values N(0, 0.5^2), positions drawn until all
four surrounding points are sea.  H and H^T are torch gather / index_add (test
harness, not the operator).  The autograd gradient must equal
V_H^T H^T (H V_H v - y) built from the hand-written adjoint, agree with a
central difference, and a steepest-descent step with the exact line search of
the quadratic must lower J."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1404_5756_gb300 import Plan, synth, vh  # noqa: E402

pytestmark = pytest.mark.gpu


def bilinear(w, obs, device):
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    i0 = np.minimum(np.floor(obs["x"]).astype(np.int64), nx - 2)
    j0 = np.minimum(np.floor(obs["y"]).astype(np.int64), ny - 2)
    fx, fy = obs["x"] - i0, obs["y"] - j0
    base = (obs["var"] * nz + obs["lev"]) * ny * nx
    idx = np.stack([base + j0 * nx + i0, base + j0 * nx + i0 + 1,
                    base + (j0 + 1) * nx + i0, base + (j0 + 1) * nx + i0 + 1])
    wts = np.stack([(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy])
    idx = torch.from_numpy(idx).to(device)
    wts = torch.from_numpy(wts.astype(np.float32)).to(device)

    def H(u):
        return (u.reshape(-1)[idx] * wts).sum(0)

    def Ht(r, like):
        out = torch.zeros(like.numel(), device=device, dtype=r.dtype)
        out.index_add_(0, idx.reshape(-1), (wts * r).reshape(-1))
        return out.reshape(like.shape)

    return H, Ht


@pytest.fixture(scope="module")
def problem():
    w = synth.workload(2, nz=4, nvar=2)
    obs = synth.observations(w)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=4))
    H, Ht = bilinear(w, obs, "cuda")
    yobs = torch.from_numpy(obs["value"]).cuda()
    v = torch.from_numpy(w["x"]).cuda()
    return w, plan, H, Ht, yobs, v


def test_interpolation_adjoint_pair(problem):
    w, plan, H, Ht, yobs, v = problem
    rng = np.random.default_rng(3)
    u = torch.from_numpy(rng.standard_normal(v.shape)).cuda()
    r = torch.from_numpy(rng.standard_normal(yobs.numel())).cuda()
    lhs = (H(u.float()).double() * r).sum()
    rhs = (u * Ht(r.float(), v).double()).sum()
    assert abs(lhs - rhs).item() <= 1e-5 * abs(lhs).item()


def test_gradient_is_the_adjoint_chain_and_matches_differences(problem):
    w, plan, H, Ht, yobs, v = problem

    def J(vv):
        r = H(vh(vv, plan)) - yobs
        return 0.5 * (r * r).sum()

    vv = v.clone().requires_grad_(True)
    J(vv).backward()
    with torch.no_grad():
        r = H(plan.apply(v)) - yobs
        ref = plan.apply_adjoint(Ht(r, v))
    assert torch.allclose(vv.grad, ref, rtol=0, atol=1e-5 * ref.abs().max().item())
    rng = np.random.default_rng(4)
    d = torch.from_numpy(rng.standard_normal(v.shape).astype(np.float32)).cuda()
    with torch.no_grad():
        fd = (J(v + d).double() - J(v - d).double()) / 2.0
    an = (vv.grad.double() * d.double()).sum()
    assert abs(fd.item() - an.item()) <= 1e-3 * abs(an.item())


def test_exact_line_search_step_lowers_the_cost(problem):
    w, plan, H, Ht, yobs, v = problem
    with torch.no_grad():
        r = H(plan.apply(v)) - yobs
        j0 = 0.5 * (r.double() ** 2).sum().item()
        g = plan.apply_adjoint(Ht(r, v))
        Ag = H(plan.apply(g))
        alpha = (g.double() ** 2).sum() / (Ag.double() ** 2).sum()
        r1 = H(plan.apply(v - alpha.float() * g)) - yobs
        j1 = 0.5 * (r1.double() ** 2).sum().item()
    # for a quadratic the decrease is exactly ||g||^4 / (2 ||A g||^2)
    expected = ((g.double() ** 2).sum() ** 2 / (2 * (Ag.double() ** 2).sum())).item()
    assert j1 < j0
    assert abs((j0 - j1) - expected) <= 1e-3 * expected
