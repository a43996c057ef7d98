"""Conjugate gradients on the system of Eq. "eight" in control-variable form,
(I + V_H^T H^T R^-1 H V_H) v = V_H^T H^T R^-1 d, with V_H from the library
(one CG iteration captured as a CUDA graph) against the same CG in FP64 with
the oracle's V_H.  H is bilinear interpolation at seeded observations (test
harness).  The observation precision (1e-4) makes CG need about 30
iterations: the FP64 solve's relative residual is about 1e-2 after 10 and
below 1e-8 after 30, so both solvers converge and their solutions must
agree to FP32 accuracy."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Plan, synth  # noqa: E402
from paper_1404_5756_gb300.var3d import Var3D  # noqa: E402

pytestmark = pytest.mark.gpu
RINV = 1e-4
ITERS = 30


def small_problem():
    w = synth.workload(2, nz=2, nvar=2)
    ny, nx = 96, 160
    w = dict(w, ny=ny, nx=nx, mask=w["mask"][:ny, :nx], Lx=w["Lx"][:ny, :nx],
             Ly=w["Ly"][:ny, :nx], x=np.ascontiguousarray(w["x"][:, :, :ny, :nx]))
    obs = synth.observations(w, 3000)
    i0 = np.minimum(np.floor(obs["x"]).astype(np.int64), nx - 2)
    j0 = np.minimum(np.floor(obs["y"]).astype(np.int64), ny - 2)
    fx, fy = obs["x"] - i0, obs["y"] - j0
    base = (obs["var"] * w["nz"] + obs["lev"]) * ny * nx
    idx = np.stack([base + j0 * nx + i0, base + j0 * nx + i0 + 1,
                    base + (j0 + 1) * nx + i0, base + (j0 + 1) * nx + i0 + 1])
    wts = np.stack([(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy])
    return w, obs, idx, wts


def torch_ops(idx, wts, shape):
    ti = torch.from_numpy(idx).cuda()
    tw = torch.from_numpy(wts.astype(np.float32)).cuda()
    n = int(np.prod(shape))

    def H(u):
        return (u.reshape(-1)[ti] * tw).sum(0)

    def Ht(r):
        out = torch.zeros(n, device="cuda", dtype=r.dtype)
        out.index_add_(0, ti.reshape(-1), (tw * r).reshape(-1))
        return out.reshape(shape)

    return H, Ht


def oracle_cg(w, obs, idx, wts, iters):
    shape = w["x"].shape

    def V(u, adjoint=False):
        return orc.vh(u, w["mask"], w["Lx"].astype(np.float64), w["Ly"].astype(np.float64),
                      adjoint=adjoint)

    def H(u):
        return (u.reshape(-1)[idx] * wts).sum(0)

    def Ht(r):
        out = np.zeros(int(np.prod(shape)))
        np.add.at(out, idx.reshape(-1), (wts * r).reshape(-1))
        return out.reshape(shape)

    def A(p):
        return p + V(Ht(RINV * H(V(p))), adjoint=True)

    d = obs["value"].astype(np.float64)
    b = V(Ht(RINV * d), adjoint=True)
    v = np.zeros(shape)
    r = b.copy()
    p = r.copy()
    rr = (r * r).sum()
    for _ in range(iters):
        Ap = A(p)
        alpha = rr / (p * Ap).sum()
        v += alpha * p
        r -= alpha * Ap
        rr_new = (r * r).sum()
        p = r + (rr_new / rr) * p
        rr = rr_new
    return v, np.linalg.norm(b - A(v)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def setup():
    w, obs, idx, wts = small_problem()
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=w["nz"]))
    H, Ht = torch_ops(idx, wts, w["x"].shape)
    d = torch.from_numpy(obs["value"]).cuda()
    rinv = torch.full_like(d, RINV)
    prob = Var3D(plan, H, Ht, rinv, d, w["x"].shape)
    return w, obs, idx, wts, prob


def test_cg_with_graphed_iterations_matches_fp64_oracle_cg(setup):
    w, obs, idx, wts, prob = setup
    v_ref, res_ref = oracle_cg(w, obs, idx, wts, ITERS)
    assert res_ref < 1e-8                       # the FP64 solve has converged
    v = prob.solve(ITERS).double().cpu().numpy()
    err = np.abs(v - v_ref).max() / np.abs(v_ref).max()
    assert err <= 1e-4, err
    # the GPU solution satisfies the normal equations to FP32 accuracy
    b = prob.rhs()
    Av = prob.apply_A(torch.from_numpy(v.astype(np.float32)).cuda(), torch.empty_like(b))
    assert ((b - Av).norm() / b.norm()).item() <= 1e-4


def test_graphed_and_eager_iterations_agree_and_cost_decreases(setup):
    w, obs, idx, wts, prob = setup
    v_g, hist = prob.solve(8, graph=True, record=True)
    v_e = prob.solve(8, graph=False)
    assert torch.allclose(v_g, v_e, rtol=0, atol=1e-5 * v_e.abs().max().item())
    assert hist[-1] < 0.1 * hist[0]                          # the residual shrinks
    costs = [prob.cost(prob.solve(k, graph=False)) for k in range(0, 6)]
    assert all(b < a for a, b in zip(costs, costs[1:]))      # CG lowers J every step
    assert prob.plan.status() == 0
