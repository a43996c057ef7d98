"""Thin ctypes binding over librfvh.so (include/rfvh.h), same names.

Argument marshalling only: every step of the filter runs in the CUDA library.
PyTorch provides device memory and the current stream.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librfvh.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "rfvh.h")

RF_OK, RF_EINVAL, RF_ENOMEM, RF_ECUDA, RF_ETIMEOUT, RF_EUNSUPPORTED = range(6)
RF_NORM_GAUSS_PEAK, RF_NORM_UNIT_SUM = 0, 1
RF_FLAG_Q_CORRECTED = 1
RF_FLAG_COAST_CONSTANT = 2
RF_FLAG_COAST_CARRIED = 4


class rf_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("mask_nz", ctypes.c_int64),
                ("L_nz", ctypes.c_int64)]


class rf_options(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("iters", ctypes.c_int),
                ("img_factor", ctypes.c_double), ("norm", ctypes.c_int),
                ("flags", ctypes.c_int), ("chunk", ctypes.c_int),
                ("tile", ctypes.c_int)]


class RFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)}")


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions include/rfvh.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(rf_\w+)\s*\(", text, flags=re.M)


def load(build_if_missing: bool = False):
    """Load librfvh.so (building it first only if asked); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        from . import build as _b
        _b.build()
    lib = ctypes.CDLL(LIB_PATH)
    i, i64, vp, d = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    lib.rf_options_default.argtypes = [ctypes.POINTER(rf_options)]
    lib.rf_coeffs.argtypes = [ctypes.POINTER(rf_grid), i, pp, pp, pp,
                              ctypes.POINTER(rf_options), vp, ctypes.POINTER(vp)]
    lib.rf_apply.argtypes = [vp, pp, pp, i, vp]
    lib.rf_apply_adjoint.argtypes = [vp, pp, pp, i, vp]
    lib.rf_apply_host.argtypes = [vp, pp, pp, i, i, vp]
    lib.rf_apply_static.argtypes = [vp, pp, pp, i, i, vp]
    lib.rf_plan_tune.argtypes = [vp, i, vp]
    lib.rf_plan_tune_batch.argtypes = [vp, i, vp]
    lib.rf_plan_status.argtypes = [vp]
    lib.rf_plan_set_wait_limit.argtypes = [vp, i]
    lib.rf_plan_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i),
                                 ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.rf_plan_destroy.argtypes = [vp]
    lib.rf_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.rf_graph_create.argtypes = [vp, pp, pp, i, i, ctypes.POINTER(vp)]
    lib.rf_graph_launch.argtypes = [vp, vp]
    lib.rf_graph_destroy.argtypes = [vp]
    lib.rf_status_string.argtypes = [i]
    lib.rf_status_string.restype = ctypes.c_char_p
    for name in ("rf_options_default", "rf_coeffs", "rf_apply", "rf_apply_adjoint",
                 "rf_apply_host", "rf_apply_static", "rf_plan_tune", "rf_plan_tune_batch",
                 "rf_plan_status", "rf_plan_set_wait_limit",
                 "rf_plan_info", "rf_plan_destroy", "rf_plan_describe", "rf_graph_create", "rf_graph_launch",
                 "rf_graph_destroy"):
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().rf_status_string(code).decode()
    except Exception:   # library not loadable: still report the code
        return f"rf_status {code}"


def check(code: int, where: str) -> None:
    if code != RF_OK:
        raise RFError(code, where)


def ptr_array(ptrs) -> ctypes.Array:
    arr = (ctypes.c_void_p * max(len(ptrs), 1))()
    for k, p in enumerate(ptrs):
        arr[k] = p
    return arr


def rf_options_default() -> rf_options:
    o = rf_options()
    check(load().rf_options_default(ctypes.byref(o)), "rf_options_default")
    return o


def rf_coeffs(grids, masks, Lxs, Lys, opt, stream) -> ctypes.c_void_p:
    """grids: list of rf_grid; masks/Lxs/Lys: device pointers (int)."""
    lib = load()
    g = (rf_grid * len(grids))(*grids)
    plan = ctypes.c_void_p()
    rc = lib.rf_coeffs(g, len(grids), ptr_array(masks), ptr_array(Lxs),
                       ptr_array(Lys), ctypes.byref(opt) if opt is not None else None,
                       ctypes.c_void_p(stream), ctypes.byref(plan))
    check(rc, "rf_coeffs")
    return plan


def rf_apply(plan, ins, outs, nvar, stream, adjoint=False) -> None:
    lib = load()
    fn = lib.rf_apply_adjoint if adjoint else lib.rf_apply
    check(fn(plan, ptr_array(ins), ptr_array(outs), int(nvar), ctypes.c_void_p(stream)),
          "rf_apply_adjoint" if adjoint else "rf_apply")


def rf_apply_adjoint(plan, ins, outs, nvar, stream) -> None:
    rf_apply(plan, ins, outs, nvar, stream, adjoint=True)


def rf_apply_host(plan, ins, outs, nvar, adjoint, stream) -> None:
    check(load().rf_apply_host(plan, ptr_array(ins), ptr_array(outs), int(nvar),
                               int(bool(adjoint)), ctypes.c_void_p(stream)),
          "rf_apply_host")


def rf_plan_tune(plan, nvar, stream) -> None:
    check(load().rf_plan_tune(plan, int(nvar), ctypes.c_void_p(stream)), "rf_plan_tune")


def rf_plan_tune_batch(plan, nvar, stream) -> None:
    check(load().rf_plan_tune_batch(plan, int(nvar), ctypes.c_void_p(stream)),
          "rf_plan_tune_batch")


def rf_plan_status(plan) -> int:
    return load().rf_plan_status(plan)


def rf_plan_set_wait_limit(plan, polls: int) -> None:
    check(load().rf_plan_set_wait_limit(plan, int(polls)), "rf_plan_set_wait_limit")


def rf_plan_info(plan):
    """(points per variable, domains, device bytes, kernel launches)."""
    pts, nd, nb, nl = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    check(load().rf_plan_info(plan, ctypes.byref(pts), ctypes.byref(nd),
                              ctypes.byref(nb), ctypes.byref(nl)), "rf_plan_info")
    return pts.value, nd.value, nb.value, nl.value


def rf_plan_describe(plan) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    check(load().rf_plan_describe(plan, buf, len(buf)), "rf_plan_describe")
    return buf.value.decode()


def rf_plan_destroy(plan) -> None:
    check(load().rf_plan_destroy(plan), "rf_plan_destroy")


def rf_graph_create(plan, ins, outs, nvar, adjoint) -> ctypes.c_void_p:
    g = ctypes.c_void_p()
    check(load().rf_graph_create(plan, ptr_array(ins), ptr_array(outs), int(nvar),
                                 int(bool(adjoint)), ctypes.byref(g)), "rf_graph_create")
    return g


def rf_graph_launch(graph, stream) -> None:
    check(load().rf_graph_launch(graph, ctypes.c_void_p(stream)), "rf_graph_launch")


def rf_graph_destroy(graph) -> None:
    check(load().rf_graph_destroy(graph), "rf_graph_destroy")
