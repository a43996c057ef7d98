"""ctypes shim over the FP64 CPU oracle in rf_oracle.c.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check of
__graft_entry__ and by the CPU-baseline leg of bench.py, never by the product
package.  It shares no code with the CUDA library.

Functions follow the paper (Farina et al., Sec. 3 and Appendix A): see the
header of rf_oracle.c for the step-by-step description and the pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RF_ORACLE_SRC / RF_ORACLE_LIB point the shim at another source and library:
# the mutation test builds copies with planted mistakes this way, to show
# that the pins catch them.
_SRC = os.environ.get("RF_ORACLE_SRC") or os.path.join(_HERE, "rf_oracle.c")
_LIB = os.environ.get("RF_ORACLE_LIB") or os.path.join(_HERE, "librforacle.so")

NORM_GAUSS_PEAK = 0
NORM_UNIT_SUM = 1
COAST_ZERO = 0        # imaginary sea points carry zero (the paper's reading)
COAST_CONSTANT = 1    # imaginary sea points carry the adjacent sea value
COAST_CARRIED = 2     # imaginary sea points keep their values across 1st-RF iterations


def build(force: bool = False) -> str:
    """Compile rf_oracle.c with gcc (no FMA contraction) into librforacle.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off",
                           "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", _SRC,
                           "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        vp = ctypes.c_void_p
        lib.orc_q_of_sigma.argtypes = [d]
        lib.orc_q_of_sigma.restype = d
        lib.orc_rf3_coeffs.argtypes = [d, i, i, vp, vp, vp]
        lib.orc_rf3_coeffs.restype = None
        lib.orc_rf1_coeffs.argtypes = [d, i, i, vp, vp]
        lib.orc_rf1_coeffs.restype = None
        lib.orc_line.argtypes = [i, i, i, d, i, i, i, i64, vp, vp, vp, vp]
        lib.orc_line.restype = i
        lib.orc_vh.argtypes = [i, i, i, d, i, i, i, i64, i64, i64, i64, vp, i64,
                               vp, vp, i64, vp, vp]
        lib.orc_vh.restype = i
        lib.orc_n_imaginary.argtypes = [d, d]
        lib.orc_n_imaginary.restype = i64
        lib.orc_set_threads.argtypes = [i]
        lib.orc_set_threads.restype = i
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def n_imaginary(img_factor: float, sigma: float) -> int:
    """Imaginary points the oracle puts at a coast of length scale sigma
    (img_factor = inf: the cut of the infinite imaginary sea)."""
    return int(_load().orc_n_imaginary(float(img_factor), float(sigma)))


def set_threads(n: int) -> int:
    """Threads of vh()'s loop over (variable, level) slices (OpenMP; 1 by
    default).  Results do not depend on it."""
    return int(_load().orc_set_threads(int(n)))


def q_of_sigma(sigma: float) -> float:
    """q of the q-corrected 3rd-RF: the filter of Theorem 3.1 taken at q has
    impulse-response variance sigma^2."""
    return float(_load().orc_q_of_sigma(float(sigma)))


def rf3_coeffs(sigma: float, norm: int = NORM_GAUSS_PEAK, qcorr: bool = False):
    """Theorem 3.1 coefficients: returns (a[4], alpha[3], beta); qcorr takes
    the a_j at q(sigma) (beta still normalised with sigma)."""
    lib = _load()
    a = np.zeros(4)
    al = np.zeros(3)
    b = np.zeros(1)
    lib.orc_rf3_coeffs(float(sigma), int(norm), int(bool(qcorr)), _ptr(a), _ptr(al), _ptr(b))
    return a, al, float(b[0])


def rf1_coeffs(sigma: float, K: int, norm: int = NORM_GAUSS_PEAK):
    """1st-RF coefficients from Hayden's relation: returns (alpha, beta)."""
    lib = _load()
    al = np.zeros(1)
    b = np.zeros(1)
    lib.orc_rf1_coeffs(float(sigma), int(K), int(norm), _ptr(al), _ptr(b))
    return float(al[0]), float(b[0])


def line(x, sigma, mask=None, *, order: int = 3, iters: int = 1,
         adjoint: bool = False, img_factor: float = 3.0,
         norm: int = NORM_GAUSS_PEAK, qcorr: bool = False,
         coast: int = COAST_ZERO) -> np.ndarray:
    """Apply one 1-D filter G (or G^T) to the line x.  coast: COAST_ZERO
    (imaginary points carry zero), COAST_CONSTANT (the adjacent sea value) or
    COAST_CARRIED (zero at first, then their own values from iteration to
    iteration)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    sig = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, np.float64), (n,)))
    m = (np.ones(n, np.uint8) if mask is None
         else np.ascontiguousarray(mask, dtype=np.uint8))
    out = np.zeros(n)
    rc = lib.orc_line(order, iters, int(adjoint), float(img_factor), norm, int(bool(qcorr)),
                      int(coast), n,
                      _ptr(m), _ptr(sig), _ptr(x), _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_line failed with code {rc}")
    return out


def vh(field, mask, Lx, Ly, *, order: int = 3, iters: int = 1,
       adjoint: bool = False, img_factor: float = 3.0,
       norm: int = NORM_GAUSS_PEAK, qcorr: bool = False,
       coast: int = COAST_ZERO) -> np.ndarray:
    """V_H = G_y G_x (adjoint: G_x^T G_y^T) on a field [nvar][nz][ny][nx].

    field may also be [nz][ny][nx] or [ny][nx]; mask is [mask_nz][ny][nx]
    or [ny][nx]; Lx, Ly are [L_nz][ny][nx] or [ny][nx] (grid units).
    """
    lib = _load()
    f = np.asarray(field, dtype=np.float64)
    shape = f.shape
    while f.ndim < 4:
        f = f[None]
    nvar, nz, ny, nx = f.shape
    f = np.ascontiguousarray(f)

    def lev(a, dtype):
        a = np.asarray(a, dtype=dtype)
        if a.ndim == 2:
            a = a[None]
        return np.ascontiguousarray(a)

    m = lev(mask, np.uint8)
    lx = lev(Lx, np.float64)
    ly = lev(Ly, np.float64)
    out = np.zeros_like(f)
    rc = lib.orc_vh(order, iters, int(adjoint), float(img_factor), norm, int(bool(qcorr)),
                    int(coast), nx, ny, nz, nvar, _ptr(m), m.shape[0], _ptr(lx), _ptr(ly),
                    lx.shape[0], _ptr(f), _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_vh failed with code {rc}")
    return out.reshape(shape)
