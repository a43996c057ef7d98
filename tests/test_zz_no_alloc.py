"""The allocation-free entry point rf_apply_static, called through the C ABI.

It serves callers that must not allocate device memory when they apply the
operator (a framework that owns every allocation through its own pool, code
that cannot afford the implicit synchronisation of cudaMalloc/cudaFree, or a
loop that may not allocate after start-up).  Its scratch is a static device
array inside the library instead of plan-grown memory.  Its results must
match rf_apply / rf_apply_adjoint within the parity tolerance, call after
call (the array keeps the previous call's contents).  This file is collected
last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1404_5756_gb300 import Options, Plan, _lib, synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


def apply_static(plan, x, out, nvar, adjoint):
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    xs = x if isinstance(x, (list, tuple)) else [x]
    outs = out if isinstance(out, (list, tuple)) else [out]
    return lib.rf_apply_static(plan.handle, _lib.ptr_array([t.data_ptr() for t in xs]),
                               _lib.ptr_array([t.data_ptr() for t in outs]), nvar, int(adjoint),
                               stream)


@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
def test_static_matches_rf_apply_on_two_calls(order, K):
    w = synth.workload(2, nz=2, nvar=2)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=2), Options(order=order, iters=K))
    x = torch.from_numpy(w["x"]).cuda()
    for adjoint in (False, True):
        ref = plan.apply_adjoint(x) if adjoint else plan.apply(x)
        for _ in range(2):
            out = torch.full_like(x, float("nan"))
            assert apply_static(plan, x, out, 2, adjoint) == _lib.RF_OK
            torch.cuda.synchronize()
            err = ((out - ref).abs().max() / ref.abs().max()).item()
            assert err <= TOL
    assert plan.status() == _lib.RF_OK


def test_static_rejects_scratch_beyond_its_size():
    """A checkerboard mask makes every sea point a segment end: 32 slices of
    32768 ends per direction need 3.1 M scratch floats, above the 2^21 the
    static array holds, so the call is refused before any launch.  Four
    slices fit: the call with the most scratch records per line that passes
    the check must match rf_apply."""
    n = 256
    j, i = np.mgrid[0:n, 0:n]
    mask = ((i + j) % 2).astype(np.uint8)
    L = np.full((n, n), 3.0, np.float32)
    plan = Plan(dict(mask=mask, Lx=L, Ly=L, nz=1))
    x = torch.zeros((32, 1, n, n), device="cuda")
    assert apply_static(plan, x, x, 32, False) == _lib.RF_EINVAL
    rng = np.random.default_rng(12)
    x4 = torch.from_numpy(rng.standard_normal((4, 1, n, n)).astype(np.float32)).cuda()
    for adjoint in (False, True):
        out = torch.full_like(x4, float("nan"))
        assert apply_static(plan, x4, out, 4, adjoint) == _lib.RF_OK
        torch.cuda.synchronize()
        ref = plan.apply_adjoint(x4) if adjoint else plan.apply(x4)
        assert ((out - ref).abs().max() / ref.abs().max()).item() <= TOL


def test_static_allocates_nothing():
    """After a first call, further calls leave the plan's device bytes and
    the device's free memory unchanged, and a call captured into a CUDA graph
    (where an allocation would fail the capture) replays correctly."""
    w = synth.workload(2, nz=2, nvar=2)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=2), Options(order=1, iters=5))
    x = torch.from_numpy(w["x"]).cuda()
    out = torch.empty_like(x)
    ref = plan.apply(x)
    assert apply_static(plan, x, out, 2, False) == _lib.RF_OK
    torch.cuda.synchronize()
    bytes0 = plan.info()[2]
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert apply_static(plan, x, out, 2, False) == _lib.RF_OK
    torch.cuda.synchronize()
    assert plan.info()[2] == bytes0
    assert torch.cuda.mem_get_info()[0] == free0
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        out.fill_(float("nan"))
        g.capture_begin()
        rc = apply_static(plan, x, out, 2, False)
        g.capture_end()
    torch.cuda.current_stream().wait_stream(s)
    assert rc == _lib.RF_OK
    g.replay()
    torch.cuda.synchronize()
    assert ((out - ref).abs().max() / ref.abs().max()).item() <= TOL


def test_static_two_domains():
    """A plan of two domains of different sizes (the per-domain size check
    and the in[d] / out[d] loop) matches rf_apply domain by domain."""
    doms = synth.ragged_domains(2, scale=0.05, max_levels=3)
    specs = [dict(mask=d["mask"], Lx=d["Lx"], Ly=d["Ly"], nz=d["nz"]) for d in doms]
    plan = Plan(specs, Options(order=3))
    rng = np.random.default_rng(13)
    xs = [torch.from_numpy(rng.standard_normal((2, d["nz"]) + np.asarray(d["mask"]).shape)
                           .astype(np.float32)).cuda() for d in doms]
    assert xs[0].shape != xs[1].shape
    for adjoint in (False, True):
        refs = plan.apply_adjoint(xs) if adjoint else plan.apply(xs)
        outs = [torch.full_like(t, float("nan")) for t in xs]
        assert apply_static(plan, xs, outs, 2, adjoint) == _lib.RF_OK
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            assert ((o - r).abs().max() / r.abs().max()).item() <= TOL
