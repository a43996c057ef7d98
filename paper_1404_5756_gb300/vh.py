"""PyTorch-facing API of the V_H recursive-filter operator.

`Plan` wraps an rf_plan (coefficients, segments and boundary maps for one or
more domains); `Plan.apply` / `Plan.apply_adjoint` call rf_apply /
rf_apply_adjoint on torch CUDA tensors on the current stream, and
`VhFunction` makes V_H differentiable with the hand-written adjoint as its
backward (the transposed filter the 3D-VAR gradient needs, Eq. "eight" of
the paper).  Tensors only carry memory and streams; all arithmetic runs in
librfvh.so.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


@dataclass
class Options:
    order: int = 3          # 3: Theorem 3.1 filter; 1: Sec. 3.1 filter
    iters: int = 1          # K (1 for order 3)
    img_factor: float = 3.0
    norm: int = _lib.RF_NORM_GAUSS_PEAK
    qcorr: bool = False     # q-corrected 3rd-RF: impulse variance sigma^2
    # imaginary points carry "zero", the edge value ("constant"), or zero at
    # first and then their own values across the 1st-RF iterations ("carried")
    coast: str = "zero"

    def to_c(self) -> _lib.rf_options:
        flag = {"zero": 0, "constant": _lib.RF_FLAG_COAST_CONSTANT,
                "carried": _lib.RF_FLAG_COAST_CARRIED}
        if self.coast not in flag:
            raise ValueError(f"coast must be 'zero', 'constant' or 'carried', not {self.coast!r}")
        o = _lib.rf_options_default()
        o.order, o.iters = int(self.order), int(self.iters)
        o.img_factor, o.norm = float(self.img_factor), int(self.norm)
        o.flags = (_lib.RF_FLAG_Q_CORRECTED if self.qcorr else 0) | flag[self.coast]
        return o


def _stream_handle(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _as_levels(a: torch.Tensor) -> torch.Tensor:
    return a.unsqueeze(0) if a.dim() == 2 else a


class Plan:
    """Plan for a batch of domains.

    domains: list of dicts (or one dict) with keys mask [mask_nz][ny][nx]
    (or [ny][nx]) uint8, Lx and Ly [L_nz][ny][nx] (or [ny][nx]) float32, and
    nz (levels).  Arrays may be numpy or torch; they are copied to `device`.
    """

    def __init__(self, domains, options: Options | None = None,
                 device: str | torch.device = "cuda"):
        if isinstance(domains, dict):
            domains = [domains]
        self.options = options or Options()
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("Plan needs a CUDA device: the filter has no CPU path")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        _lib.load()
        grids, masks, lxs, lys, keep = [], [], [], [], []
        self.shapes = []
        for d in domains:
            m = _as_levels(torch.as_tensor(np.asarray(d["mask"]) if not torch.is_tensor(d["mask"]) else d["mask"]))
            lx = _as_levels(torch.as_tensor(d["Lx"]))
            ly = _as_levels(torch.as_tensor(d["Ly"]))
            m = m.to(self.device, torch.uint8).contiguous()
            lx = lx.to(self.device, torch.float32).contiguous()
            ly = ly.to(self.device, torch.float32).contiguous()
            nz = int(d.get("nz", max(m.shape[0], lx.shape[0])))
            ny, nx = int(m.shape[-2]), int(m.shape[-1])
            if tuple(lx.shape[-2:]) != (ny, nx) or lx.shape != ly.shape:
                raise ValueError("mask, Lx and Ly must share the horizontal grid")
            grids.append(_lib.rf_grid(nx, ny, nz, int(m.shape[0]), int(lx.shape[0])))
            masks.append(m.data_ptr())
            lxs.append(lx.data_ptr())
            lys.append(ly.data_ptr())
            keep += [m, lx, ly]
            self.shapes.append((nz, ny, nx))
        with torch.cuda.device(self.device):
            self._plan = _lib.rf_coeffs(grids, masks, lxs, lys, self.options.to_c(),
                                        _stream_handle(self.device))
        del keep

    # ------------------------------------------------------------------ info
    @property
    def handle(self):
        return self._plan

    def info(self):
        """(points per variable, domains, device bytes owned, kernel launches)."""
        return _lib.rf_plan_info(self._plan)

    def tune(self, nvar: int) -> None:
        """Time the tile-kernel launch shapes for `nvar` variables and keep the
        fastest (rf_plan_tune); synchronises the current stream."""
        with torch.cuda.device(self.device):
            _lib.rf_plan_tune(self._plan, nvar, _stream_handle(self.device))

    def tune_batch(self, nvar: int) -> None:
        """Tune only the multi-domain launches (rf_plan_tune_batch)."""
        with torch.cuda.device(self.device):
            _lib.rf_plan_tune_batch(self._plan, nvar, _stream_handle(self.device))

    def describe(self) -> str:
        """The plan's chunking and the launch configurations chosen so far."""
        return _lib.rf_plan_describe(self._plan)

    def status(self) -> int:
        return _lib.rf_plan_status(self._plan)

    def set_wait_limit(self, polls: int) -> None:
        """Bound of the kernels' device-side waits in polls (0: give up at
        once, which makes rf_plan_status report RF_ETIMEOUT)."""
        _lib.rf_plan_set_wait_limit(self._plan, polls)

    def close(self):
        if getattr(self, "_plan", None):
            _lib.rf_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- apply
    def _check(self, xs, nvar):
        if len(xs) != len(self.shapes):
            raise ValueError(f"expected {len(self.shapes)} domain tensors, got {len(xs)}")
        for x, (nz, ny, nx) in zip(xs, self.shapes):
            if x.dtype != torch.float32 or x.device != self.device:
                raise ValueError("fields must be float32 tensors on the plan's device")
            if not x.is_contiguous() or x.numel() != nvar * nz * ny * nx:
                raise ValueError(f"field must be contiguous [nvar][{nz}][{ny}][{nx}]")

    def _run(self, x, out, adjoint):
        single = torch.is_tensor(x)
        xs = [x] if single else list(x)
        nz, ny, nx = self.shapes[0]
        nvar = xs[0].numel() // (nz * ny * nx)
        self._check(xs, nvar)
        if out is None:
            outs = [torch.empty_like(t) for t in xs]
        else:
            outs = [out] if single else list(out)
            self._check(outs, nvar)
        with torch.cuda.device(self.device):
            _lib.rf_apply(self._plan, [t.data_ptr() for t in xs],
                          [t.data_ptr() for t in outs], nvar,
                          _stream_handle(self.device), adjoint=adjoint)
        return outs[0] if single else outs

    def apply(self, x, out=None):
        """V_H x (x: one tensor [nvar][nz][ny][nx] or a list, one per domain)."""
        return self._run(x, out, False)

    def apply_adjoint(self, x, out=None):
        """V_H^T x."""
        return self._run(x, out, True)

    def graph(self, x, out, adjoint: bool = False) -> "Graph":
        """CUDA graph of one application on fixed buffers (rf_graph_create):
        replaying it computes out = V_H x (adjoint: V_H^T x) for the current
        contents of x."""
        single = torch.is_tensor(x)
        xs = [x] if single else list(x)
        outs = [out] if single else list(out)
        nz, ny, nx = self.shapes[0]
        nvar = xs[0].numel() // (nz * ny * nx)
        self._check(xs, nvar)
        self._check(outs, nvar)
        with torch.cuda.device(self.device):
            g = _lib.rf_graph_create(self._plan, [t.data_ptr() for t in xs],
                                     [t.data_ptr() for t in outs], nvar, adjoint)
        return Graph(self, g, xs + outs)

    def apply_host(self, xs, outs, nvar: int, adjoint: bool = False):
        """End-to-end call on host (ideally pinned) CPU tensors: the library
        copies in, applies, copies out and synchronises."""
        single = torch.is_tensor(xs)
        xs = [xs] if single else list(xs)
        outs = [outs] if single else list(outs)
        for t in xs + outs:
            if t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError("apply_host takes contiguous float32 CPU tensors")
        with torch.cuda.device(self.device):
            _lib.rf_apply_host(self._plan, [t.data_ptr() for t in xs],
                               [t.data_ptr() for t in outs], nvar, adjoint,
                               _stream_handle(self.device))


class Graph:
    """An executable CUDA graph of one V_H (or V_H^T) application.  Holds
    its plan and buffers so they outlive it."""

    def __init__(self, plan: Plan, handle, tensors):
        self.plan = plan
        self._g = handle
        self._keep = tensors

    def launch(self) -> None:
        with torch.cuda.device(self.plan.device):
            _lib.rf_graph_launch(self._g, _stream_handle(self.plan.device))

    def close(self) -> None:
        if getattr(self, "_g", None):
            _lib.rf_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VhFunction(torch.autograd.Function):
    """y = V_H x with backward g -> V_H^T g (the hand-written adjoint)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.apply(x.contiguous())

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        return ctx.plan.apply_adjoint(g.contiguous()), None


def vh(x: torch.Tensor, plan: Plan) -> torch.Tensor:
    return VhFunction.apply(x, plan)
