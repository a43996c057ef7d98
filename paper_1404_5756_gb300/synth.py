"""Seeded synthetic inputs shaped like the paper's ocean grids.

This module only draws inputs (fields, land masks, length-scale fields); it
holds none of the filter's arithmetic, so both the CUDA path and the FP64
oracle can be fed from it.  All randomness is NumPy PCG64 seeded with
1404 + the workload id, generated on the host.

Workloads (the paper's data sets are not available, so these stand in for
them with the same shapes):
  1. 256 x 128, one level, all sea, uniform L = 10 (the impulse setup of
     Sec. 3.1, Fig. 1, in 2-D);
  2. regional basin 1024 x 384 x 72 levels, T and S (Mediterranean
     configuration of Sec. 4 scaled down), ~30 % land, L smooth in [5, 40];
  3. global 1440 x 1080 x 75 levels (the 1/4 degree configuration of Sec. 5),
     ~30 % land, L latitude-like from 4 (poles) to 30 (equator);
  5. ragged batch of 64 independent domains.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1404


def rng_for(workload: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + workload))


def smooth_noise(rng: np.random.Generator, ny: int, nx: int, std: float) -> np.ndarray:
    """N(0,1) noise blurred by a periodic Gaussian of `std` grid points (FFT)."""
    w = rng.standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    transfer = np.exp(-2.0 * (np.pi * std) ** 2 * (kx * kx + ky * ky))
    return np.real(np.fft.ifft2(np.fft.fft2(w) * transfer))


def land_mask(rng: np.random.Generator, ny: int, nx: int, blur: float,
              land_frac: float) -> np.ndarray:
    """uint8 mask, 1 = sea, 0 = land; exactly the `land_frac` lowest values of
    a smoothed noise field are land, which gives coastlines and islands."""
    if land_frac <= 0.0:
        return np.ones((ny, nx), np.uint8)
    f = smooth_noise(rng, ny, nx, blur)
    order = np.argsort(f, axis=None, kind="stable")
    m = np.ones(ny * nx, np.uint8)
    m[order[: int(round(land_frac * ny * nx))]] = 0
    return m.reshape(ny, nx)


def length_field(rng: np.random.Generator, ny: int, nx: int, blur: float,
                 lo: float, hi: float) -> np.ndarray:
    """Smooth random length scale (grid units) mapped affinely onto [lo, hi]."""
    f = smooth_noise(rng, ny, nx, blur)
    f = (f - f.min()) / max(f.max() - f.min(), 1e-300)
    return (lo + (hi - lo) * f).astype(np.float32)


def latitude_length(ny: int, nx: int, lo: float = 4.0, hi: float = 30.0) -> np.ndarray:
    """L_j = lo + (hi - lo) cos^2(pi (j/(ny-1) - 1/2)): long scales in the
    tropics, short at the poles (Sec. 5 describes this pattern)."""
    j = np.arange(ny, dtype=np.float64)
    t = j / max(ny - 1, 1) - 0.5
    row = lo + (hi - lo) * np.cos(np.pi * t) ** 2
    return np.repeat(row[:, None], nx, axis=1).astype(np.float32)


def normal_field(rng: np.random.Generator, shape) -> np.ndarray:
    return rng.standard_normal(shape, dtype=np.float32)


def workload(wid: int, *, nz: int | None = None, nvar: int | None = None,
             fields: bool = True) -> dict:
    """Grid, mask, length scales and (optionally) input fields of a workload.

    Returns a dict with nx, ny, nz, nvar, mask [ny][nx] u8, Lx, Ly [ny][nx]
    f32 and, if `fields`, x [nvar][nz][ny][nx] f32 drawn N(0,1).
    `nz`/`nvar` override the level/variable count (smaller parity cases).
    """
    rng = rng_for(wid)
    if wid == 1:
        nx, ny, nz0, nv0 = 256, 128, 1, 1
        mask = np.ones((ny, nx), np.uint8)
        L = np.full((ny, nx), 10.0, np.float32)
    elif wid in (2, 4):
        nx, ny, nz0, nv0 = 1024, 384, 72, 2
        mask = land_mask(rng, ny, nx, 12.0, 0.30)
        L = length_field(rng, ny, nx, 48.0, 5.0, 40.0)
    elif wid == 3:
        nx, ny, nz0, nv0 = 1440, 1080, 75, 1
        mask = land_mask(rng, ny, nx, 16.0, 0.30)
        L = latitude_length(ny, nx)
    else:
        raise ValueError(f"unknown workload {wid}")
    nz = nz0 if nz is None else nz
    nvar = nv0 if nvar is None else nvar
    out = dict(wid=wid, nx=nx, ny=ny, nz=nz, nvar=nvar, mask=mask, Lx=L,
               Ly=L.copy())
    if fields:
        out["x"] = normal_field(rng, (nvar, nz, ny, nx))
    return out


def impulse(ny: int, nx: int, j: int, i: int) -> np.ndarray:
    x = np.zeros((1, 1, ny, nx), np.float32)
    x[0, 0, j, i] = 1.0
    return x


def ragged_domains(n: int = 64, *, wid: int = 5, scale: float = 1.0,
                   max_levels: int = 75) -> list[dict]:
    """Ragged batch: nx ~ U{128..2048}, ny ~ U{64..1024}, nz ~ U{1..75},
    land fraction ~ U[0, 0.4] (blur max(nx,ny)/64), L in [3, 40].
    `scale` < 1 shrinks every domain (parity cases the oracle finishes fast)."""
    rng = rng_for(wid)
    doms = []
    for _ in range(n):
        nx = int(rng.integers(128, 2049))
        ny = int(rng.integers(64, 1025))
        nz = int(rng.integers(1, max_levels + 1))
        land = float(rng.uniform(0.0, 0.4))
        if scale != 1.0:
            nx = max(8, int(nx * scale))
            ny = max(8, int(ny * scale))
            nz = max(1, int(nz * scale))
        blur = max(nx, ny) / 64.0
        mask = land_mask(rng, ny, nx, blur, land)
        L = length_field(rng, ny, nx, 4.0 * blur, 3.0, 40.0)
        doms.append(dict(nx=nx, ny=ny, nz=nz, mask=mask, Lx=L, Ly=L.copy()))
    return doms


def observations(w: dict, nobs: int = 50_000, *, wid: int = 4, sd: float = 0.5) -> dict:
    """Seeded observation set for the 3D-VAR cost of workload `w`: each
    observation draws a variable and a level uniformly and a continuous
    position (x, y) uniformly, redrawn until the four grid points around it
    are sea; its value is N(0, sd^2).  Returns var, lev (int64), x, y
    (float64 grid coordinates) and value (float32)."""
    rng = rng_for(wid)
    mask = np.asarray(w["mask"]).astype(bool)
    ny, nx = mask.shape[-2:]
    var = rng.integers(0, w["nvar"], nobs)
    lev = rng.integers(0, w["nz"], nobs)
    xs = np.empty(nobs)
    ys = np.empty(nobs)
    todo = np.arange(nobs)
    while todo.size:
        x = rng.uniform(0.0, nx - 1.0, todo.size)
        y = rng.uniform(0.0, ny - 1.0, todo.size)
        i = np.minimum(x.astype(np.int64), nx - 2)
        j = np.minimum(y.astype(np.int64), ny - 2)
        ok = mask[j, i] & mask[j, i + 1] & mask[j + 1, i] & mask[j + 1, i + 1]
        xs[todo[ok]] = x[ok]
        ys[todo[ok]] = y[ok]
        todo = todo[~ok]
    value = rng.normal(0.0, sd, nobs).astype(np.float32)
    return dict(var=var, lev=lev, x=xs, y=ys, value=value)
