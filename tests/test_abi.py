"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/rfvh.h declares, and rejects bad
arguments before queueing any GPU work."""
import ctypes

import pytest

from paper_1404_5756_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    return _lib.load(build_if_missing=True)


def test_header_declares_the_boundary():
    names = _lib.declared_functions()
    for n in ["rf_coeffs", "rf_apply", "rf_apply_adjoint", "rf_plan_status",
              "rf_plan_destroy", "rf_status_string", "rf_options_default",
              "rf_apply_host", "rf_plan_info", "rf_plan_tune"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _lib.declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(6):
        s = _lib.status_string(code)
        assert s.startswith("RF_")
    assert "unknown" in _lib.status_string(99)


def test_options_default(lib):
    o = _lib.rf_options_default()
    assert (o.order, o.iters, o.img_factor, o.norm, o.flags) == (3, 1, 3.0, 0, 0)
    assert lib.rf_options_default(None) == _lib.RF_EINVAL


def _coeffs(lib, grid, opt, masks=(1,), lx=(1,), ly=(1,), nd=1, out=True):
    g = (_lib.rf_grid * max(nd, 1))(*([grid] * max(nd, 1)))
    plan = ctypes.c_void_p()
    return lib.rf_coeffs(g, nd, _lib.ptr_array(list(masks)), _lib.ptr_array(list(lx)),
                         _lib.ptr_array(list(ly)),
                         ctypes.byref(opt) if opt is not None else None, None,
                         ctypes.byref(plan) if out else None)


def test_rf_coeffs_rejects_bad_arguments(lib):
    ok_grid = _lib.rf_grid(16, 8, 2, 1, 1)
    opt = _lib.rf_options_default()
    E = _lib.RF_EINVAL
    assert _coeffs(lib, ok_grid, opt, nd=0) == E
    assert _coeffs(lib, ok_grid, opt, out=False) == E
    assert _coeffs(lib, ok_grid, opt, masks=(None,)) == E
    assert _coeffs(lib, ok_grid, opt, lx=(None,)) == E
    for bad in [_lib.rf_grid(0, 8, 2, 1, 1), _lib.rf_grid(16, 8, 0, 1, 1),
                _lib.rf_grid(16, 8, 3, 2, 1), _lib.rf_grid(16, 8, 3, 1, 2)]:
        assert _coeffs(lib, bad, opt) == E

    def with_(**kw):
        o = _lib.rf_options_default()
        for k, v in kw.items():
            setattr(o, k, v)
        return o
    for o in [with_(order=2), with_(order=3, iters=2), with_(order=1, iters=0),
              with_(img_factor=-1.0), with_(img_factor=float("-inf")),
              with_(img_factor=float("nan")), with_(norm=5), with_(flags=8),
              with_(chunk=-1), with_(tile=-3),
              with_(flags=_lib.RF_FLAG_COAST_CONSTANT | 8),
              with_(order=1, iters=5,
                    flags=_lib.RF_FLAG_COAST_CONSTANT | _lib.RF_FLAG_COAST_CARRIED),
              with_(order=1, iters=5, flags=_lib.RF_FLAG_Q_CORRECTED),
              with_(order=1, iters=5,
                    flags=_lib.RF_FLAG_Q_CORRECTED | _lib.RF_FLAG_COAST_CONSTANT)]:
        assert _coeffs(lib, ok_grid, o) == E


def test_rf_coeffs_refuses_what_this_build_does_not_provide(lib):
    """Valid requests the library does not build return RF_EUNSUPPORTED
    before any GPU work: chunk-length and tile-shape overrides (the kernels
    derive both from the line length), and the infinite imaginary sea with
    constant-extension coasts."""
    ok_grid = _lib.rf_grid(16, 8, 2, 1, 1)
    U = _lib.RF_EUNSUPPORTED

    def with_(**kw):
        o = _lib.rf_options_default()
        for k, v in kw.items():
            setattr(o, k, v)
        return o
    for o in [with_(chunk=32), with_(tile=4), with_(chunk=1, tile=1),
              with_(img_factor=float("inf"), flags=_lib.RF_FLAG_COAST_CONSTANT)]:
        assert _coeffs(lib, ok_grid, o) == U


def test_apply_rejects_bad_arguments(lib):
    E = _lib.RF_EINVAL
    arr = _lib.ptr_array([1])
    assert lib.rf_apply(None, arr, arr, 1, None) == E
    assert lib.rf_apply_adjoint(None, arr, arr, 1, None) == E
    assert lib.rf_apply_host(None, arr, arr, 1, 0, None) == E
    assert lib.rf_plan_status(None) == E
    assert lib.rf_plan_set_wait_limit(None, 0) == E
    assert lib.rf_plan_tune(None, 1, None) == E
    assert lib.rf_plan_info(None, None, None, None, None) == E
    assert lib.rf_plan_destroy(None) == _lib.RF_OK


def test_product_path_has_no_oracle_dependency():
    """The product package never imports the oracle."""
    import os
    import re
    pkg = os.path.dirname(_lib.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert not re.search(r"\boracle\b\s*import|import\s+oracle|from\s+oracle",
                                     text), f


def test_python_options_map_to_the_c_flags(lib):
    """Options -> rf_options: the q-correction and the coast treatment become
    RF_FLAG_Q_CORRECTED, RF_FLAG_COAST_CONSTANT and RF_FLAG_COAST_CARRIED, and
    the C header carries the same values the binding uses."""
    from paper_1404_5756_gb300 import Options
    hdr = open(_lib.HEADER).read()
    assert "RF_FLAG_Q_CORRECTED = 1" in hdr and "RF_FLAG_COAST_CONSTANT = 2" in hdr
    assert "RF_FLAG_COAST_CARRIED = 4" in hdr
    cases = [(dict(), 0), (dict(qcorr=True), _lib.RF_FLAG_Q_CORRECTED),
             (dict(coast="constant"), _lib.RF_FLAG_COAST_CONSTANT),
             (dict(coast="carried"), _lib.RF_FLAG_COAST_CARRIED),
             (dict(qcorr=True, coast="constant"),
              _lib.RF_FLAG_Q_CORRECTED | _lib.RF_FLAG_COAST_CONSTANT)]
    for kw, flags in cases:
        o = Options(**kw).to_c()
        assert o.flags == flags
        assert (o.order, o.iters, o.img_factor, o.norm) == (3, 1, 3.0, 0)
    o = Options(order=1, iters=5, img_factor=2.5, norm=_lib.RF_NORM_UNIT_SUM).to_c()
    assert (o.order, o.iters, o.img_factor, o.norm, o.flags) == (1, 5, 2.5, 1, 0)
    with pytest.raises(ValueError):
        Options(coast="reflect").to_c()


def test_plan_refuses_a_cpu_device():
    torch = pytest.importorskip("torch")
    from paper_1404_5756_gb300 import Plan
    mask = torch.ones(4, 5, dtype=torch.uint8)
    L = torch.full((4, 5), 2.0)
    with pytest.raises(ValueError):
        Plan(dict(mask=mask, Lx=L, Ly=L, nz=1), device="cpu")
