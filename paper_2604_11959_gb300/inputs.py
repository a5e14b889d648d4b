"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke
check: terrain heights at the lattice nodes, the stratified initial state and
the fixed time step.  This module holds none of the EB method's arithmetic
(no geometry, fluxes or redistribution); both the CUDA path and the CPU oracle
take its arrays as plain inputs.

Shapes follow the C ABI: nodal heights are (ny+1, nx+1) with the last row and
column repeating the first (periodic), state fields are (nz_g, ny, nx) with
x fastest, nz_g = nz for rho, rho*theta, rho*u, rho*v and nz+1 for rho*w.

Workloads are shaped like the paper's hill-flow cases (Sec. 6: the Witch of
Agnesi ridge and a three-dimensional hill), with a Gaussian random field of
k^-3 spectrum standing in for real terrain.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# constants of the reference state (Sec. 2): gas constant, heat capacity,
# reference pressure, gravity, surface potential temperature, buoyancy freq.
R_D = 287.0
C_P = 1004.5
P00 = 1.0e5
GRAV = 9.81
THETA_S = 300.0
N_BV = 0.01


def _periodic_nodes(f, nx, ny):
    """f evaluated on the (ny+1, nx+1) node lattice, last row/col = first."""
    h = np.empty((ny + 1, nx + 1), dtype=np.float64)
    h[:ny, :nx] = f
    h[:ny, nx] = f[:, 0]
    h[ny, :] = h[0, :]
    return h


def woa_ridge(nx, ny, Lx=1.0, hp=0.1, a=0.1):
    """Witch-of-Agnesi ridge h = hp / (1 + ((x - Lx/2)/a)^2), uniform in y."""
    x = np.arange(nx) * (Lx / nx)
    row = hp / (1.0 + ((x - 0.5 * Lx) / a) ** 2)
    return _periodic_nodes(np.broadcast_to(row, (ny, nx)), nx, ny)


def gaussian_hill(nx, ny, Lx=1.0, Ly=1.0, h0=0.15, sigma=0.08, centre=(0.5, 0.5)):
    """Gaussian hill h = h0 exp(-r^2 / (2 sigma^2)) about ``centre``."""
    x = np.arange(nx) * (Lx / nx)
    y = np.arange(ny) * (Ly / ny)
    r2 = (x[None, :] - centre[0]) ** 2 + (y[:, None] - centre[1]) ** 2
    return _periodic_nodes(h0 * np.exp(-r2 / (2.0 * sigma ** 2)), nx, ny)


def grf_terrain(nx, ny, seed, hmax=0.2, slope=-3.0):
    """Periodic Gaussian random field with power spectral density |k|^slope
    (amplitude |k|^(slope/2)) on integer wavenumbers, zero mean mode,
    rescaled to [0, hmax]."""
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(nx, d=1.0 / nx)
    ky = np.fft.fftfreq(ny, d=1.0 / ny)
    kk = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    amp = np.zeros_like(kk)
    amp[kk > 0] = kk[kk > 0] ** (slope / 2.0)
    coef = (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))) * amp
    f = np.real(np.fft.ifft2(coef))
    f = (f - f.min()) / (f.max() - f.min()) * hmax
    return _periodic_nodes(f, nx, ny)


def plant_tiny_cells(h, nx, ny, nz, Lz, count, seed, eps=1e-6, min_sep=4):
    """Flatten ``count`` seeded, well separated columns: their four corner
    nodes are set to eps*dz below the top of the cell holding the highest of
    them, which leaves a cell with volume fraction about eps.  Returns the new
    heights and the planted (i, j, k) list."""
    core = np.array(h[:ny, :nx], dtype=np.float64)
    dz = Lz / nz
    rng = np.random.default_rng(seed)
    picked = []
    tries = 0
    while len(picked) < count and tries < 100000:
        tries += 1
        i, j = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        far = all(max(min(abs(i - pi), nx - abs(i - pi)), min(abs(j - pj), ny - abs(j - pj))) >= min_sep
                  for (pi, pj, _) in picked)
        if not far:
            continue
        corners = [((i + a) % nx, (j + b) % ny) for a in (0, 1) for b in (0, 1)]
        top = max(core[cj, ci] for ci, cj in corners)
        k0 = int(np.floor(top / dz))
        if k0 + 2 > nz:
            continue
        for ci, cj in corners:
            core[cj, ci] = (k0 + 1) * dz - eps * dz
        picked.append((i, j, k0))
    return _periodic_nodes(core, nx, ny), picked


# --------------------------------------------------------------------------
# stratified reference state and initial condition
# --------------------------------------------------------------------------

def reference_profile(z):
    """Hydrostatic reference of a constant-N atmosphere: theta0, rho0 at z
    (metres; the domain's length unit is read as metres)."""
    z = np.asarray(z, dtype=np.float64)
    theta0 = THETA_S * np.exp(N_BV ** 2 * z / GRAV)
    exner = 1.0 + GRAV ** 2 / (C_P * THETA_S * N_BV ** 2) * (np.exp(-N_BV ** 2 * z / GRAV) - 1.0)
    p0 = P00 * exner ** (C_P / R_D)
    rho0 = p0 / (R_D * exner * theta0)
    return theta0, rho0


def cell_reference(nz, Lz):
    """rho0 and rho0*theta0 at the cell-centre levels (k + 1/2) dz."""
    zc = (np.arange(nz) + 0.5) * (Lz / nz)
    th0, r0 = reference_profile(zc)
    return r0, r0 * th0


def initial_state(nx, ny, nz, Lz, u0=(1.0, 0.0, 0.0), pert=0.0, seed=0):
    """Stratified state at rest relative to a uniform wind u0:
    rho = rho0(z_c), rho*theta = rho0 theta0(z_c), rho*u = rho0(z_c) u0 on the
    u faces of the same level, rho*v likewise, rho*w = rho0 w0 on interior w
    levels and 0 on the wall levels k = 0, nz.  With pert > 0 every field gets
    seeded cell-wise noise of relative amplitude ``pert`` (momenta relative to
    rho0 * max(|u0|, 1))."""
    r0, rt0 = cell_reference(nz, Lz)
    shape = (nz, ny, nx)
    rho = np.broadcast_to(r0[:, None, None], shape).copy()
    rhot = np.broadcast_to(rt0[:, None, None], shape).copy()
    rhou = rho * u0[0]
    rhov = rho * u0[1]
    rhow = np.zeros((nz + 1, ny, nx))
    rw = 0.5 * (r0[:-1] + r0[1:])
    rhow[1:nz] = (rw * u0[2])[:, None, None]
    if pert > 0.0:
        rng = np.random.default_rng(seed)
        scale = max(abs(u0[0]), abs(u0[1]), abs(u0[2]), 1.0)
        rho = rho * (1.0 + pert * rng.uniform(-1, 1, shape))
        rhot = rhot * (1.0 + pert * rng.uniform(-1, 1, shape))
        rhou = rhou + pert * scale * r0[:, None, None] * rng.uniform(-1, 1, shape)
        rhov = rhov + pert * scale * r0[:, None, None] * rng.uniform(-1, 1, shape)
        noise = rng.uniform(-1, 1, (nz + 1, ny, nx))
        noise[0] = 0.0
        noise[nz] = 0.0
        rzw = np.concatenate([[r0[0]], rw, [r0[-1]]])
        rhow = rhow + pert * scale * rzw[:, None, None] * noise
    return {"rho": np.ascontiguousarray(rho), "rhotheta": np.ascontiguousarray(rhot),
            "rhou": np.ascontiguousarray(rhou), "rhov": np.ascontiguousarray(rhov),
            "rhow": np.ascontiguousarray(rhow)}


def background_momentum(nz, Lz, u0=1.0, z_calm=None, ramp=None):
    """Per-level background momenta (rho0 u_bg(z), 0) at the cell-centre
    levels, the horizontal wind the states below are built around: the wind
    u0 along x everywhere, or (z_calm, ramp given) calm below z_calm and
    ramping linearly to u0 over ``ramp``, as in ``sheltered_state``."""
    r0, _ = cell_reference(nz, Lz)
    zc = (np.arange(nz) + 0.5) * (Lz / nz)
    prof = np.ones(nz) if z_calm is None else np.clip((zc - z_calm) / ramp, 0.0, 1.0)
    return r0 * u0 * prof, np.zeros(nz)


def sheltered_state(nx, ny, nz, Lx, Ly, Lz, z_calm, ramp, u0=1.0, pert=1e-2, seed=0, modes=3):
    """Stratified state for long runs: the wind u0 blows along x above
    z_calm + ramp, is calm below z_calm (which lies above the terrain) and
    ramps linearly in between; every field carries a smooth seeded
    perturbation made of Fourier modes with wavenumbers up to ``modes`` per
    direction (relative amplitude ``pert``), so no wave shorter than
    L/modes is excited."""
    r0, rt0 = cell_reference(nz, Lz)
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    zc = (np.arange(nz) + 0.5) / nz
    zw = np.arange(nz + 1) / nz

    def smooth(zs):
        f = np.zeros((len(zs), ny, nx))
        for _ in range(2 * modes):
            kx, ky, kz = (int(v) for v in rng.integers(0, modes + 1, 3))
            px, py, pz = rng.uniform(0, 2 * np.pi, 3)
            a = rng.uniform(-1, 1)
            f += a * (np.cos(2 * np.pi * kz * zs + pz)[:, None, None] * np.cos(2 * np.pi * ky * y + py)[None, :, None]
                      * np.cos(2 * np.pi * kx * x + px)[None, None, :])
        return f / (2 * modes)

    ramp_c = np.clip(((np.arange(nz) + 0.5) * (Lz / nz) - z_calm) / ramp, 0.0, 1.0)
    shape = (nz, ny, nx)
    rho = r0[:, None, None] * (1.0 + 0.1 * pert * smooth(zc))
    rhot = rt0[:, None, None] * (1.0 + pert * smooth(zc))
    rhou = r0[:, None, None] * (u0 * ramp_c[:, None, None] + pert * u0 * smooth(zc))
    rhov = r0[:, None, None] * (pert * u0 * smooth(zc)) + np.zeros(shape)
    rw = np.concatenate([[r0[0]], 0.5 * (r0[:-1] + r0[1:]), [r0[-1]]])
    rhow = rw[:, None, None] * (pert * u0 * smooth(zw))
    rhow[0] = 0.0
    rhow[nz] = 0.0
    return {"rho": np.ascontiguousarray(rho), "rhotheta": np.ascontiguousarray(rhot),
            "rhou": np.ascontiguousarray(rhou), "rhov": np.ascontiguousarray(rhov),
            "rhow": np.ascontiguousarray(rhow)}


def fixed_dt(nx, ny, nz, Lx, Ly, Lz, u0=(1.0, 0.0, 0.0), cfl=0.5):
    """Time step held fixed over a run: CFL / (|u|/dx + |v|/dy + |w|/dz) of the
    uniform wind."""
    rate = abs(u0[0]) * nx / Lx + abs(u0[1]) * ny / Ly + abs(u0[2]) * nz / Lz
    return cfl / rate


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    steps: int
    Lx: float = 1.0
    Ly: float = 1.0
    Lz: float = 0.5
    terrain: str = "gaussian"
    seed: int = 0
    hmax: float = 0.15
    tiny: int = 0
    sigma: float = 0.08

    def heights(self):
        if self.terrain == "woa":
            return woa_ridge(self.nx, self.ny, self.Lx)
        if self.terrain == "gaussian":
            return gaussian_hill(self.nx, self.ny, self.Lx, self.Ly, h0=self.hmax, sigma=self.sigma)
        if self.terrain == "grf":
            h = grf_terrain(self.nx, self.ny, self.seed, hmax=self.hmax)
            if self.tiny:
                h, _ = plant_tiny_cells(h, self.nx, self.ny, self.nz, self.Lz, self.tiny, self.seed + 1)
            return h
        if self.terrain == "flat":
            return np.full((self.ny + 1, self.nx + 1), self.hmax)
        raise ValueError(self.terrain)

    def dt(self):
        return fixed_dt(self.nx, self.ny, self.nz, self.Lx, self.Ly, self.Lz)

    def state(self, kind="uniform", pert=0.0, seed=0):
        """'uniform': the wind u0 = 1 everywhere (short runs); 'sheltered': calm
        below the terrain top, u0 = 1 above a ramp of 8 cells (long runs)."""
        if kind == "uniform":
            return initial_state(self.nx, self.ny, self.nz, self.Lz, pert=pert, seed=seed)
        dz = self.Lz / self.nz
        return sheltered_state(self.nx, self.ny, self.nz, self.Lx, self.Ly, self.Lz,
                               z_calm=self.hmax + dz, ramp=8 * dz, pert=pert if pert else 1e-2, seed=seed)

    def cells(self):
        return self.nx * self.ny * self.nz

    def references(self, kind="uniform"):
        """Per-level profiles (rho0, rho0 theta0, rho0 u_bg, rho0 v_bg) of the
        state ``kind``: the stratified reference and the background wind the
        state is built around (the wind of ``state(kind)`` without its
        perturbations)."""
        r0, rt0 = cell_reference(self.nz, self.Lz)
        if kind == "uniform":
            ru, rv = background_momentum(self.nz, self.Lz)
        else:
            dz = self.Lz / self.nz
            ru, rv = background_momentum(self.nz, self.Lz, z_calm=self.hmax + dz, ramp=8 * dz)
        return r0, rt0, ru, rv


WOA_32 = Workload("woa-ridge-32x32x16", 32, 32, 16, 10, terrain="woa", hmax=0.1)
HILL_256 = Workload("gaussian-hill-256x256x128", 256, 256, 128, 100, terrain="gaussian", hmax=0.15)
GRF_512 = Workload("grf-k3-512x512x256", 512, 512, 256, 50, terrain="grf", seed=3, hmax=0.2, tiny=16)
GRF_192 = Workload("grf-k3-192x192x96", 192, 192, 96, 10, terrain="grf", seed=4, hmax=0.15)


def anelastic_state(w: Workload, seed=0):
    """The sheltered wind of ``w`` with the density at the reference profile
    (the anelastic model's rho = rho0)."""
    U = w.state("sheltered", seed=seed)
    U = {f: np.array(v, copy=True) for f, v in U.items()}
    rho0 = cell_reference(w.nz, w.Lz)[0]
    U["rho"] = np.broadcast_to(rho0[:, None, None], U["rho"].shape).copy()
    return U


def ensemble_members():
    """64 uneven Gaussian-hill instances: nx = ny = 64 (1 + b mod 4),
    nz = 32 (1 + floor(b/4) mod 2), hill height 0.05 + 0.15 u1 and width
    0.05 + 0.10 u2 from default_rng(1000 + b)."""
    out = []
    for b in range(64):
        n = 64 * (1 + b % 4)
        nz = 32 * (1 + (b // 4) % 2)
        rng = np.random.default_rng(1000 + b)
        u1, u2 = rng.uniform(), rng.uniform()
        out.append((n, n, nz, 0.05 + 0.15 * u1, 0.05 + 0.10 * u2))
    return out
