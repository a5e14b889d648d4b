"""Training and evaluation of the projection's warm-start network.

Orchestration only: every sample comes from the library's solver
(``eb_project_sample``) and every update from its kernels
(``eb_unet_train_step``); this module chooses terrains, states and the order
of the steps.

Training domains have the cell size of the target problem (the network is
fully convolutional: trained on 96 x 96 x 48 cells, it runs on
192 x 192 x 96 cells of the same size), seeded k^-3 random terrain, and the
anelastic initial state (sheltered wind, density at the reference) with seeded
perturbations.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import eb, inputs

# (cin, cout, kernel size) of the library's network, in parameter order
LAYERS = [(2, 16, 3), (16, 16, 3), (16, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3),
          (96, 32, 3), (32, 32, 3), (48, 16, 3), (16, 16, 3), (16, 1, 1)]


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, std sqrt(2 / fan_in), zero biases; the head layer
    starts small so the first guesses are close to zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (ci, co, k) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (ci * k ** 3)) * (0.1 if l == len(LAYERS) - 1 else 1.0)
        parts.append(rng.standard_normal(co * ci * k ** 3) * std)
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


@dataclasses.dataclass
class Recipe:
    nx: int = 96
    ny: int = 96
    nz: int = 48
    dx: float = 1.0 / 192.0
    hmax_frac: float = 0.3     # terrain height over the domain height
    terrains: int = 48
    states_per_terrain: int = 8
    epochs: int = 12
    lr: float = 1e-3
    rtol: float = 1e-10
    seed: int = 100


def workload(r: Recipe, t: int, nx=None, ny=None, nz=None) -> inputs.Workload:
    nx, ny, nz = nx or r.nx, ny or r.ny, nz or r.nz
    return inputs.Workload(f"terrain-{t}", nx, ny, nz, 1, Lx=nx * r.dx, Ly=ny * r.dx, Lz=nz * r.dx, terrain="grf",
                           seed=r.seed + t, hmax=r.hmax_frac * nz * r.dx)


def geometry(w: inputs.Workload, preconditioner: str = "jacobi"):
    refs = inputs.cell_reference(w.nz, w.Lz)
    g = eb.Geometry(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, torch.from_numpy(w.heights()).cuda(), precision="mixed",
                    ref_rho=torch.from_numpy(refs[0]).cuda(), ref_rhotheta=torch.from_numpy(refs[1]).cuda())
    eb.set_preconditioner(g, preconditioner)
    return g, refs


def state(w, refs, seed):
    return eb.device_state(inputs.anelastic_state(w, seed=seed), "mixed", refs)


def target_scale(r: Recipe) -> float:
    """The spread of the solution in units of rms(rhs) dx^2 on a few pilot
    problems; training targets are divided by it (order one)."""
    vals = []
    for t in range(3):
        w = workload(r, 10_000 + t)
        g, refs = geometry(w)
        _, tt, m, _ = eb.project_sample(g, state(w, refs, t), w.dt(), 1.0, rtol=1e-8)
        vals.append(float(tt[m > 0].std()))
        g.close()
    return float(np.median(vals))


def make_dataset(r: Recipe, scale: float, first_terrain: int = 0, terrains: int | None = None):
    """Samples (input, target, mask) on the GPU and the cold-start iteration
    count of each (multigrid-preconditioned solves: the samples are the same
    converged solutions, found faster)."""
    data, iters = [], []
    for t in range(first_terrain, first_terrain + (terrains or r.terrains)):
        w = workload(r, t)
        g, refs = geometry(w, "mg")
        for s in range(r.states_per_terrain):
            x, tt, m, it = eb.project_sample(g, state(w, refs, 1000 * t + s), w.dt(), scale, rtol=r.rtol)
            data.append((x, tt, m))
            iters.append(it)
        g.close()
    return data, iters


def train(r: Recipe, data, log=None) -> eb.UNet:
    net = eb.UNet(r.nx, r.ny, r.nz)
    net.set_params(init_params(r.seed))
    rng = np.random.default_rng(r.seed)
    steps = 0
    t0 = time.perf_counter()
    for ep in range(r.epochs):
        lr = r.lr * (0.5 * (1.0 + np.cos(np.pi * ep / r.epochs)))   # cosine decay per epoch
        losses = []
        for q in rng.permutation(len(data)):
            x, t, m = data[q]
            want = steps % 50 == 0
            l = net.train_step(x, t, m, lr, want_loss=want)
            if want:
                losses.append(l)
            steps += 1
        if log:
            log(f"epoch {ep}: lr {lr:.2e}, loss {np.mean(losses):.4e}, {time.perf_counter() - t0:.1f} s")
    torch.cuda.synchronize()
    return net


def compare(geom, net_params, w, refs, seed, scale, rtol=1e-10):
    """Cold (zero) and warm (network) starts of the same projection:
    (cold iterations, warm iterations, max momentum difference relative to
    the momentum scale)."""
    net = eb.UNet(w.nx, w.ny, w.nz)
    net.set_params(net_params)
    U = state(w, refs, seed)
    A = {f: U[f].clone() for f in U}
    B = {f: U[f].clone() for f in U}
    dt = w.dt()
    it_c, res_c = eb.project(geom, A, dt, rtol=rtol)
    it_w, res_w = eb.project_warm(geom, net, B, dt, scale, rtol=rtol)
    ms = max(float(A[f].abs().max()) for f in ("rhou", "rhov", "rhow"))
    diff = max(float((A[f] - B[f]).abs().max()) for f in ("rhou", "rhov", "rhow")) / ms
    net.close()
    return it_c, it_w, res_c, res_w, diff


def guess_error(net: eb.UNet, data, block: int = 8):
    """Relative error of the network's guess on samples (input, target, mask):
    over all fluid cells, and on the smooth part (means over blocks of
    block^3 cells, the modes conjugate gradients converge on last), as the
    median over the samples.  Measurement only: the guess itself comes from
    the library's forward pass."""
    fine, smooth = [], []
    pool = torch.nn.functional.avg_pool3d
    for x, t, m in data:
        y = net.forward(x)
        e, tm = (y - t) * m, t * m
        fine.append(float(e.norm() / tm.norm()))
        es = pool(e[None, None], block, ceil_mode=True)
        ts = pool(tm[None, None], block, ceil_mode=True)
        smooth.append(float(es.norm() / ts.norm()))
    return float(np.median(fine)), float(np.median(smooth))


def sequence(geom, net_params, w, refs, seed, scale, nsteps=4, rtol=1e-10):
    """Projections of consecutive forward-Euler anelastic steps (provisional
    momenta from eb_step with the density at the reference, then the
    projection) from a projected initial state, each solved from a zero
    start, from the previous step's solution and from the network's guess.
    Returns one (zero, previous, network) iteration triple per step (previous
    is None on the first).  The converged projections agree to the solver's
    tolerance; the zero-start one advances the sequence."""
    net = eb.UNet(w.nx, w.ny, w.nz)
    net.set_params(net_params)
    dt = w.dt()
    S = state(w, refs, seed)
    eb.project(geom, S, dt, rtol=rtol)
    phi_prev = None
    rows = []
    for _ in range(nsteps):
        P = eb.step(geom, S, dt, 1)
        P["rho"].zero_()   # the anelastic density is the reference
        A = {f: P[f].clone() for f in P}
        phi = torch.empty(geom.shape(0), dtype=torch.float64, device="cuda")
        it0, _ = eb.project(geom, A, dt, rtol=rtol, phi=phi)
        itp = None
        if phi_prev is not None:
            B = {f: P[f].clone() for f in P}
            itp, _ = eb.project(geom, B, dt, rtol=rtol, phi0=phi_prev)
        C = {f: P[f].clone() for f in P}
        itw, _ = eb.project_warm(geom, net, C, dt, scale, rtol=rtol)
        rows.append((it0, itp, itw))
        phi_prev, S = phi, A
    net.close()
    return rows
