"""x-slab decomposition of one periodic domain over several ranks (one GPU
each): the multi-GPU form of the step.

Every CV's update reads the state and the geometry of CVs a bounded number
of columns away (the third-order face stencils, the averaged masses, the
redistribution neighbourhoods and least-squares stencils: seven columns per
stage, and the set-up tables three columns more), and the geometry of a
column depends only on its own lattice nodes.  So a rank that owns columns
[x0, x1) of the domain holds them with `halo` columns on either side, builds
the geometry of that extended slab from the true nodal heights, and before
every step copies its neighbours' edge columns into its halo: its owned
columns then advance exactly as in the single domain, bit for bit, while the
halo (whose stencils run off the slab) is overwritten at the next exchange.
A halo of 12 columns covers a forward-Euler step, 24 a three-stage step.

The exchange goes through ``torch.distributed`` point-to-point operations
(NCCL between GPUs, gloo between CPU processes) or, for ranks held by one
process, through plain copies (``exchange_local``).  The stepping itself is
the caller's: on GPUs the library's ``eb.step`` on the slab's geometry handle.
This module holds no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")

HALO_EULER = 12   # columns of halo per forward-Euler step between exchanges
HALO_RK3 = 24     # per three-stage step


class Slabs:
    """Column ranges of rank ``rank`` of ``world`` in an nx-column periodic
    domain, the owned columns split as evenly as possible."""

    def __init__(self, nx: int, world: int, rank: int, halo: int):
        if world < 1 or not 0 <= rank < world:
            raise ValueError("rank must lie in [0, world)")
        self.nx, self.world, self.rank, self.halo = int(nx), int(world), int(rank), int(halo)
        bounds = [(q * self.nx) // self.world for q in range(self.world + 1)]
        self.bounds = bounds
        self.x0, self.x1 = bounds[rank], bounds[rank + 1]
        if min(bounds[q + 1] - bounds[q] for q in range(self.world)) < self.halo and self.world > 1:
            raise ValueError("every slab needs at least `halo` owned columns")
        self.width = self.x1 - self.x0            # owned columns
        self.ext = self.width + 2 * self.halo     # columns held

    def columns(self) -> np.ndarray:
        """Global column index of every held column (periodic)."""
        return (np.arange(self.x0 - self.halo, self.x1 + self.halo)) % self.nx

    def heights(self, h: np.ndarray) -> np.ndarray:
        """Nodal heights of the held slab, (ny + 1, ext + 1): the true heights
        of its lattice nodes (the last node column is the slab's right edge,
        not a copy of its first)."""
        nodes = np.arange(self.x0 - self.halo, self.x1 + self.halo + 1) % self.nx
        return np.ascontiguousarray(h[:, nodes])

    def scatter(self, a):
        """The held columns of a global field (..., nx) -> (..., ext)."""
        return a[..., self.columns()]

    def interior(self, a):
        """The owned columns of a held field (..., ext) -> (..., width)."""
        return a[..., self.halo:self.halo + self.width]

    # ---- exchange -------------------------------------------------------
    def _neighbours(self):
        return (self.rank - 1) % self.world, (self.rank + 1) % self.world

    def exchange(self, U: dict, dist) -> None:
        """Fill the halo of every field of U (torch tensors (..., ext)) from
        the neighbouring ranks through torch.distributed: the left halo from
        the left neighbour's last owned columns, the right halo from the
        right neighbour's first owned columns."""
        import torch
        if self.world == 1:
            exchange_local([self], [U])
            return
        left, right = self._neighbours()
        H = self.halo
        for f in FIELDS:
            a = U[f]
            send_l = a[..., H:2 * H].contiguous()                 # my first owned columns, to the left
            send_r = a[..., self.width:self.width + H].contiguous()   # my last owned columns, to the right
            recv_l = torch.empty_like(send_l)
            recv_r = torch.empty_like(send_r)
            ops = [dist.P2POp(dist.isend, send_l, left), dist.P2POp(dist.irecv, recv_r, right),
                   dist.P2POp(dist.isend, send_r, right), dist.P2POp(dist.irecv, recv_l, left)]
            for r in dist.batch_isend_irecv(ops):
                r.wait()
            a[..., :H] = recv_l
            a[..., H + self.width:] = recv_r


def exchange_local(slabs, states) -> None:
    """The exchange of ``Slabs.exchange`` for ranks held by one process:
    slabs[q] and states[q] (dicts of fields (..., ext), numpy arrays or
    torch tensors) of every rank, in rank order."""
    n = len(slabs)
    for q, (s, U) in enumerate(zip(slabs, states)):
        L, R = states[(q - 1) % n], states[(q + 1) % n]
        sl, sr = slabs[(q - 1) % n], slabs[(q + 1) % n]
        H = s.halo
        for f in FIELDS:
            U[f][..., :H] = L[f][..., sl.width:sl.width + H]
            U[f][..., H + s.width:] = R[f][..., H:2 * H]


def advance(slabs: Slabs, U: dict, nsteps: int, step_one, dist=None):
    """nsteps steps of the held state U: before each, the exchange (through
    dist, or a periodic copy for a single rank), then ``step_one(U) -> U``
    (one step of the method on the slab).  Returns the new held state."""
    for _ in range(int(nsteps)):
        slabs.exchange(U, dist)
        U = step_one(U)
    return U
