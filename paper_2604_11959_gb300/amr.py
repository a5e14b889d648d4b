"""Two-level static refinement with one refined x-patch (Sec. 4.3).

The coarse level covers the whole periodic domain; its geometry is merged
from the fine level's cells (``Geometry.coarse``), so coarse volumes and
areas are sums of fine ones everywhere, and under the patch in particular.
The fine level exists on the patch only: the global fine columns
[x_lo, x_hi) (even bounds, the full y and z extent), held with ``halo`` fine
columns on either side (an x-window handle built from the true fine nodal
heights, as for the slab decomposition).

One step of the two levels, with the same time step on both (the fine
level's: the coarse level then runs at half its CFL number):
  1. the patch's halo takes its boundary values from the coarse state at
     time n (``prolong``: the coarse CV a fine CV lies in; on a face grid the
     mean of two coarse faces for the faces between them);
  2. both levels advance one step of Algorithm 1 (``eb.step``);
  3. the coarse CVs under the patch take the restriction of the patch's
     owned columns (``restrict``: volume- and area-weighted), the two-way
     coupling of the paper.
A halo of 12 fine columns covers a forward-Euler step, 24 a three-stage step
(the reach of one stage is seven columns): the owned columns then never see
the halo's outer edge.  The halo CVs themselves are refilled every step.
This module holds no arithmetic of the method; every operation is a kernel of
the library.
"""
from __future__ import annotations

import numpy as np

HALO_EULER = 12
HALO_RK3 = 24


class TwoLevel:
    """Coarse level (whole domain) and one fine x-patch.

    eb           the binding module (paper_2604_11959_gb300.eb)
    nx, ny, nz   fine cells of the whole domain (even); Lx, Ly, Lz its size
    h_fine       fine nodal heights, numpy (ny + 1, nx + 1)
    x_lo, x_hi   the patch's global fine columns (even)
    refs_fine, refs_coarse  per-level profiles (rho0, rho0 theta0[, background
                 rho*u, background rho*v]) of each level, numpy
    device       where the heights and profiles are handed to the binding
    """

    def __init__(self, eb, nx, ny, nz, Lx, Ly, Lz, h_fine, x_lo, x_hi, halo, precision="mixed",
                 refs_fine=None, refs_coarse=None, v_target_frac=0.5, device="cuda"):
        import torch
        if x_lo % 2 or x_hi % 2 or not 0 < x_hi - x_lo <= nx - 2 * halo:
            raise ValueError("the patch needs even bounds and room for its halo")
        self.eb, self.halo = eb, int(halo)
        self.x_lo, self.x_hi = int(x_lo), int(x_hi)
        self.width = self.x_hi - self.x_lo
        self.fine_x0 = (self.x_lo - self.halo) % nx
        cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        kw = {}
        if refs_fine is not None:
            kw = dict(ref_rho=cuda(refs_fine[0]), ref_rhotheta=cuda(refs_fine[1]))
        full = eb.Geometry(nx, ny, nz, Lx, Ly, Lz, cuda(h_fine), precision=precision, v_target_frac=v_target_frac,
                           **kw)
        ck = {}
        if refs_coarse is not None:
            ck = dict(ref_rho=cuda(refs_coarse[0]), ref_rhotheta=cuda(refs_coarse[1]))
        self.coarse = full.coarse(**ck)
        full.close()
        if refs_coarse is not None and len(refs_coarse) == 4:
            self.coarse.set_wind_reference(cuda(refs_coarse[2]), cuda(refs_coarse[3]))
        ext = self.width + 2 * self.halo
        nodes = np.arange(self.x_lo - self.halo, self.x_hi + self.halo + 1) % nx
        hp = np.ascontiguousarray(h_fine[:, nodes])
        pk = dict(kw)
        if refs_fine is not None and len(refs_fine) == 4:
            pk.update(ref_rhou=cuda(refs_fine[2]), ref_rhov=cuda(refs_fine[3]))
        self.patch = eb.Geometry(ext, ny, nz, ext * Lx / nx, Ly, Lz, cuda(hp), precision=precision,
                                 v_target_frac=v_target_frac, **pk)
        self.owned = (self.halo, self.halo + self.width)

    def fill(self, Uc, Uf):
        """Every column of the patch state from the coarse state (a start)."""
        return self.eb.prolong(self.coarse, Uc, self.patch, Uf, self.fine_x0, (0, 0))

    def step(self, Uc, Uf, dt, stages=1):
        """One step of both levels; returns the new (coarse, patch) states."""
        eb = self.eb
        eb.prolong(self.coarse, Uc, self.patch, Uf, self.fine_x0, self.owned)
        Uc1 = eb.step(self.coarse, Uc, dt, 1, stages)
        Uf1 = eb.step(self.patch, Uf, dt, 1, stages)
        eb.restrict(self.patch, self.coarse, Uf1, Uc1, self.fine_x0, self.owned)
        return Uc1, Uf1

    def close(self):
        self.patch.close()
        self.coarse.close()
