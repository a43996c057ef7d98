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
    return lib.rf_apply_static(plan.handle, _lib.ptr_array([x.data_ptr()]),
                               _lib.ptr_array([out.data_ptr()]), nvar, int(adjoint), stream)


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
    static array holds, so the call is refused before any launch."""
    n = 256
    j, i = np.mgrid[0:n, 0:n]
    mask = ((i + j) % 2).astype(np.uint8)
    L = np.full((n, n), 3.0, np.float32)
    plan = Plan(dict(mask=mask, Lx=L, Ly=L, nz=1))
    x = torch.zeros((32, 1, n, n), device="cuda")
    assert apply_static(plan, x, x, 32, False) == _lib.RF_EINVAL
    assert apply_static(plan, x[:4].contiguous(), x[:4].contiguous(), 4, False) == _lib.RF_OK
    torch.cuda.synchronize()
