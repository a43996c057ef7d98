"""V_H inside the 3D-VAR minimisation it serves.

With B = V V^T and the increment dx = V v, the quadratic cost of Eq.
"functional2" becomes, in the control variable v,

    J(v) = 1/2 v^T v + 1/2 (d - H V v)^T R^{-1} (d - H V v),

and its stationarity condition is the preconditioned system of Eq. "eight",

    (I + V^T H^T R^{-1} H V) v = V^T H^T R^{-1} d,

symmetric positive definite, which OceanVar solves with conjugate gradients
(Sec. 2.1).  Here V is the horizontal operator V_H (the other factors of
Eq. "composed" are outside this library).  H, its transpose and the
diagonal R^{-1} are supplied by the caller as tensor functions.

`Var3D.solve` runs plain CG.  One iteration (V_H, H, R^{-1}, H^T, V_H^T and
the vector updates) is captured once as a CUDA graph and replayed, so an
iteration costs one graph launch and no host synchronisation; the step
lengths stay on the device.
"""
from __future__ import annotations

from typing import Callable

import torch

from .vh import Plan


class Var3D:
    """The system of Eq. "eight" for one field [nvar][nz][ny][nx].

    plan: the V_H plan; H(u) -> observations; Ht(r) -> field (the transpose
    of H); rinv: observation-error precisions (tensor, same shape as d);
    d: the misfit y - H(x_b).  H and Ht must be made of capturable tensor
    operations on the current stream."""

    def __init__(self, plan: Plan, H: Callable, Ht: Callable, rinv: torch.Tensor,
                 d: torch.Tensor, shape):
        self.plan, self.H, self.Ht = plan, H, Ht
        self.rinv, self.d = rinv, d
        self.shape = tuple(shape)
        dev = plan.device
        self._u = torch.empty(self.shape, device=dev)   # V_H p
        self._w = torch.empty(self.shape, device=dev)   # V_H^T H^T R^-1 H V_H p

    def apply_A(self, p: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        """out = p + V_H^T H^T R^{-1} H V_H p."""
        self.plan.apply(p, out=self._u)
        self.plan.apply_adjoint(self.Ht(self.rinv * self.H(self._u)), out=self._w)
        torch.add(p, self._w, out=out)
        return out

    def rhs(self) -> torch.Tensor:
        """b = V_H^T H^T R^{-1} d."""
        return self.plan.apply_adjoint(self.Ht(self.rinv * self.d))

    def cost(self, v: torch.Tensor) -> float:
        """J(v) in float64."""
        r = self.d - self.H(self.plan.apply(v))
        return 0.5 * float((v.double() ** 2).sum() + (self.rinv.double() * r.double() ** 2).sum())

    def solve(self, iters: int, v0: torch.Tensor | None = None, graph: bool = True,
              record: bool = False):
        """Run `iters` CG iterations from v0 (default 0).  Returns v and, with
        record, the residual norms |b - A v| after each iteration (reading
        them synchronises once per iteration)."""
        dev = self.plan.device
        b = self.rhs()
        v = torch.zeros(self.shape, device=dev) if v0 is None else v0.clone()
        r = torch.empty_like(b)
        self.apply_A(v, r)
        torch.sub(b, r, out=r)
        p = r.clone()
        Ap = torch.empty_like(b)
        rr = (r * r).sum()

        def step():
            self.apply_A(p, Ap)
            alpha = rr / (p * Ap).sum()
            v.add_(alpha * p)
            r.sub_(alpha * Ap)
            rr_new = (r * r).sum()
            beta = rr_new / rr
            p.mul_(beta).add_(r)
            rr.copy_(rr_new)

        history = []
        if graph and iters > 0:
            s = torch.cuda.Stream(dev)
            s.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(s):
                # one eager call first: launch shapes and scratch are set up
                # outside the capture, so the captured calls allocate nothing
                self.apply_A(p, Ap)
            torch.cuda.current_stream(dev).wait_stream(s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            for _ in range(iters):
                g.replay()
                if record:
                    history.append(float(rr.sqrt()))
        else:
            for _ in range(iters):
                step()
                if record:
                    history.append(float(rr.sqrt()))
        return (v, history) if record else v
