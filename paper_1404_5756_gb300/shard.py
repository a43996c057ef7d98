"""Host-side sharding of V_H work across ranks (one process per GPU).

V_H = G_y G_x acts on each (variable, level) slice of each domain on its own:
no recursion crosses a level, a variable or a domain (the paper runs its
levels in parallel with OpenMP for the same reason, Section 4).  A rank can
therefore take any set of slices and filter them with no exchange at all.
This module decides which levels of which domains a rank owns and cuts the
plan inputs and fields to match; the rank then builds an ordinary plan for
its sub-domains (RankOperator).  No collective sits on the data path.

Units are (domain, level) pairs, weighted by their horizontal points; the
pairs are laid out domain after domain, level after level, and cut into
`world` contiguous pieces of nearly equal weight, so each rank gets at most
two partial domains and every piece is a contiguous level range of each
domain it touches.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Piece:
    """Levels k0 .. k0+nk-1 of domain `domain`."""
    domain: int
    k0: int
    nk: int


def _sizes(domains) -> list[tuple[int, int]]:
    out = []
    for d in domains:
        m = np.asarray(d["mask"])
        ny, nx = m.shape[-2:]
        nz = int(d.get("nz", m.shape[0] if m.ndim == 3 else 1))
        out.append((nz, int(ny) * int(nx)))
    return out


def partition(domains, world: int) -> list[list[Piece]]:
    """Per rank, the level ranges it owns.  Every (domain, level) pair lands
    on exactly one rank; the per-rank point counts differ by at most the
    points of one level."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = _sizes(domains)
    total = sum(nz * plane for nz, plane in sizes)
    ranks: list[list[Piece]] = [[] for _ in range(world)]
    acc = 0   # points assigned so far, over all ranks
    for di, (nz, plane) in enumerate(sizes):
        k = 0
        while k < nz:
            # the rank whose share [r*total/world, (r+1)*total/world) holds
            # the midpoint of level k
            mid = acc + plane // 2
            r = min(world - 1, mid * world // max(total, 1))
            # levels whose midpoints stay inside rank r's share
            hi = (r + 1) * total // world
            nk = 1
            while k + nk < nz and acc + nk * plane + plane // 2 < hi:
                nk += 1
            ranks[r].append(Piece(di, k, nk))
            acc += nk * plane
            k += nk
    return ranks


def _levels(a, k0: int, nk: int):
    a = np.asarray(a)
    if a.ndim == 2 or a.shape[0] == 1:
        return a
    return a[k0:k0 + nk]


def sub_domain(domain: dict, k0: int, nk: int) -> dict:
    """Plan inputs of levels k0 .. k0+nk-1: level-dependent masks and length
    scales are cut, 2-D ones are shared."""
    return dict(mask=_levels(domain["mask"], k0, nk), Lx=_levels(domain["Lx"], k0, nk),
                Ly=_levels(domain["Ly"], k0, nk), nz=nk)


def take(field, k0: int, nk: int):
    """Levels k0 .. k0+nk-1 of a field [nvar][nz][ny][nx] (numpy or torch),
    contiguous."""
    part = field[:, k0:k0 + nk]
    return part.contiguous() if hasattr(part, "contiguous") else np.ascontiguousarray(part)


def shard(domains, fields, rank: int, world: int):
    """(sub-domains, their fields, pieces) of `rank`: the inputs of the plan
    the rank builds and of its apply call."""
    pieces = partition(domains, world)[rank]
    subs = [sub_domain(domains[p.domain], p.k0, p.nk) for p in pieces]
    parts = [take(fields[p.domain], p.k0, p.nk) for p in pieces]
    return subs, parts, pieces


def assemble(domains, nvar: int, gathered: list[list[tuple[Piece, np.ndarray]]]):
    """Inverse of `shard` on gathered results: per domain the full field
    [nvar][nz][ny][nx], from every rank's (piece, output) pairs."""
    sizes = _sizes(domains)
    out = []
    for nz, _ in sizes:
        out.append(None)
    for per_rank in gathered:
        for p, y in per_rank:
            if out[p.domain] is None:
                nz = sizes[p.domain][0]
                out[p.domain] = np.zeros((nvar, nz) + tuple(y.shape[2:]), y.dtype)
            out[p.domain][:, p.k0:p.k0 + p.nk] = y
    return out


class RankOperator:
    """V_H on the pieces one rank owns: one Plan (on this process's GPU) over
    the rank's sub-domains, a ragged batch of level ranges, applied in one
    call with no exchange between ranks.  `parts` cuts the rank's inputs out
    of the full fields (host arrays or tensors, one [nvar][nz][ny][nx] per
    domain) onto the device; `apply` filters them and returns
    [(piece, output)] for `assemble`."""

    def __init__(self, domains, rank: int, world: int, options=None, device="cuda"):
        from .vh import Plan
        self.pieces = partition(domains, world)[rank]
        self.plan = None
        if self.pieces:
            subs = [sub_domain(domains[p.domain], p.k0, p.nk) for p in self.pieces]
            self.plan = Plan(subs, options, device=device)

    def parts(self, fields):
        """The rank's input parts on the plan's device (float32, contiguous)."""
        import torch
        out = []
        for p in self.pieces:
            x = take(fields[p.domain], p.k0, p.nk)
            x = x if torch.is_tensor(x) else torch.from_numpy(np.ascontiguousarray(x, np.float32))
            out.append(x.to(self.plan.device, torch.float32).contiguous())
        return out

    def apply(self, parts, outs=None, adjoint: bool = False):
        if not self.pieces:
            return []
        ys = self.plan._run(list(parts), None if outs is None else list(outs), adjoint)
        return list(zip(self.pieces, ys))

    def close(self):
        if self.plan is not None:
            self.plan.close()
            self.plan = None
