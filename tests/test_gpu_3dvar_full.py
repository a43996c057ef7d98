"""The 3D-VAR configuration at full size: the regional grid 1024 x 384 x 72
with T and S (56.6 M points) and 50,000 observations, J(v) = 1/2 ||H V_H v -
y||^2 (Eq. "eight", control-variable form), H bilinear.  Every observation
lies in one (variable, level) slice, so on a slice s the gradient is
V_H,s^T H_s^T (H_s V_H,s v_s - y_s): the oracle rebuilds it in FP64 on sampled
slices, and the GPU autograd gradient (FP32 operator) must match it to 1e-5
of its maximum.  The finite difference of J is taken in FP64 twice: on the
GPU with J summed in double from the FP32 operator's output (the whole
field), and on the sampled slices with J evaluated entirely in FP64 by the
oracle; J is quadratic, so the central difference has no truncation error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Plan, synth, vh  # noqa: E402

pytestmark = pytest.mark.gpu
SLICES = [(0, 0), (0, 37), (1, 11), (1, 71)]   # (variable, level) pairs checked by the oracle


def corners(w, obs):
    nx, ny = w["nx"], w["ny"]
    i0 = np.minimum(np.floor(obs["x"]).astype(np.int64), nx - 2)
    j0 = np.minimum(np.floor(obs["y"]).astype(np.int64), ny - 2)
    fx, fy = obs["x"] - i0, obs["y"] - j0
    wts = np.stack([(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy])
    return i0, j0, wts


@pytest.fixture(scope="module")
def full():
    w = synth.workload(2)
    assert w["x"].shape == (2, 72, 384, 1024)
    obs = synth.observations(w)
    assert len(obs["value"]) == 50_000
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=w["nz"]))
    i0, j0, wts = corners(w, obs)
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    base = (obs["var"] * nz + obs["lev"]) * ny * nx
    idx = np.stack([base + j0 * nx + i0, base + j0 * nx + i0 + 1,
                    base + (j0 + 1) * nx + i0, base + (j0 + 1) * nx + i0 + 1])
    idx_t = torch.from_numpy(idx).cuda()
    w64 = torch.from_numpy(wts).cuda()
    y64 = torch.from_numpy(obs["value"].astype(np.float64)).cuda()
    v = torch.from_numpy(w["x"]).cuda()

    def J64(vv):
        """J with the FP32 operator's output, H and the sum in double."""
        u = vh(vv, plan).double().reshape(-1)
        r = (u[idx_t] * w64).sum(0) - y64
        return 0.5 * (r * r).sum()

    vv = v.clone().requires_grad_(True)
    J64(vv).backward()
    torch.cuda.synchronize()
    assert plan.status() == 0
    rng = np.random.default_rng(44)
    d = rng.standard_normal(w["x"].shape).astype(np.float32)
    return dict(w=w, obs=obs, plan=plan, J64=J64, v=v, grad=vv.grad.cpu().numpy(), d=d,
                i0=i0, j0=j0, wts=wts)


def oracle_slice(f, var, lev, u):
    """H_s, J_s and the gradient of J_s on one slice, all in FP64 (oracle V_H)."""
    w, obs = f["w"], f["obs"]
    sel = (obs["var"] == var) & (obs["lev"] == lev)
    i0, j0, wts = f["i0"][sel], f["j0"][sel], f["wts"][:, sel]
    L = [np.asarray(w[k], np.float64) for k in ("Lx", "Ly")]

    def V(x, adjoint=False):
        return orc.vh(x[None, None], w["mask"], L[0], L[1], adjoint=adjoint)[0, 0]

    def H(x):
        return (wts[0] * x[j0, i0] + wts[1] * x[j0, i0 + 1] + wts[2] * x[j0 + 1, i0]
                + wts[3] * x[j0 + 1, i0 + 1])

    def Ht(r):
        out = np.zeros((w["ny"], w["nx"]))
        for k, (dj, di) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
            np.add.at(out, (j0 + dj, i0 + di), wts[k] * r)
        return out

    r = H(V(u)) - obs["value"][sel].astype(np.float64)
    return 0.5 * float(r @ r), V(Ht(r), adjoint=True), int(sel.sum())


def test_gradient_matches_the_oracle_adjoint_on_sampled_slices(full):
    g = full["grad"]
    for var, lev in SLICES:
        _, go, nobs = oracle_slice(full, var, lev, full["w"]["x"][var, lev].astype(np.float64))
        assert nobs > 0
        gs = g[var, lev]
        assert np.abs(gs - go).max() <= 1e-5 * np.abs(go).max(), (var, lev)
        # off the observed slices' sea the gradient is exactly zero at land
        assert np.all(gs[full["w"]["mask"] == 0] == 0.0)


def test_finite_differences_in_fp64(full):
    v, d, g = full["v"], full["d"], full["grad"]
    dt = torch.from_numpy(d).cuda()
    with torch.no_grad():
        fd = (full["J64"](v + dt) - full["J64"](v - dt)).item() / 2.0
    an = float((g.astype(np.float64) * d.astype(np.float64)).sum())
    assert abs(fd - an) <= 1e-4 * abs(an)
    # per sampled slice, J in FP64 end to end (oracle): exact difference
    for var, lev in SLICES:
        u = full["w"]["x"][var, lev].astype(np.float64)
        ds = d[var, lev].astype(np.float64)
        jp, _, _ = oracle_slice(full, var, lev, u + ds)
        jm, _, _ = oracle_slice(full, var, lev, u - ds)
        fd_s = (jp - jm) / 2.0
        an_s = float((g[var, lev].astype(np.float64) * ds).sum())
        assert abs(fd_s - an_s) <= 1e-5 * abs(an_s), (var, lev)
