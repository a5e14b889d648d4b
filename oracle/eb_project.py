"""FP64 CPU oracle of the anelastic projection (Sec. 2.2, Algorithm 2 step 5)
and of the anelastic step.  Test infrastructure only: the CUDA library never
imports it.

The divergence constraint div(rho0 u) = 0 is imposed on the face momenta
m = (rho0 u, rho0 v, rho0 w) with the same cut-cell finite-volume
divergence as the flux update (Eq. update-cc): for a c-cell,

    D(m)_c = sum_d ( beta_d,hi m_d,hi - beta_d,lo m_d,lo ) / delta_d,

beta the open area fractions of the cell's faces (zero on the walls z = 0,
z = Lz and on closed faces).  The pressure gradient on a face is
G(phi)_f = (phi_R - phi_L) / delta_d.  The correction m <- m* - dt G(phi)
removes the divergence when

    L phi = D(G(phi)) = D(m*) / dt,

a symmetric, negative semi-definite 7-point operator with face weights
beta / delta^2 whose null space holds the constants.  It is solved by
conjugate gradients on -L with the Jacobi preconditioner, started from
phi0 (zero by default), to the relative residual ||b - L phi|| / ||b|| <= rtol.
Covered cells (and fluid cells with every face closed) are excluded.

Arrays are numpy (nz, ny, nx), x fastest in memory; rho*w has nz + 1 levels.
Every function follows the definitions above term by term.
"""
import numpy as np


def face_weights(dom, geom):
    """Open area fractions of the low x, y, z faces of every c-cell, with the
    bottom wall closed (z = 0 carries no flux)."""
    b = np.array(geom[0]["beta"], dtype=np.float64, copy=True)
    b[2, 0] = 0.0
    return b


def _hi_z(bz):
    """beta of the high z face of every cell (the top wall is closed)."""
    out = np.zeros_like(bz)
    out[:-1] = bz[1:]
    return out


def divergence(dom, b, mu, mv, mw):
    """D(m) on every c-cell."""
    bx, by, bz = b
    fx = bx * mu
    fy = by * mv
    fz_lo = bz * mw[:-1]
    fz_hi = _hi_z(bz) * mw[1:]
    return ((np.roll(fx, -1, axis=2) - fx) / dom.dx + (np.roll(fy, -1, axis=1) - fy) / dom.dy +
            (fz_hi - fz_lo) / dom.dz)


def gradient(dom, b, phi):
    """G(phi) on the low faces of the u, v and w grids (zero on closed faces
    and on the two wall levels of w)."""
    bx, by, bz = b
    gu = np.where(bx > 0, (phi - np.roll(phi, 1, axis=2)) / dom.dx, 0.0)
    gv = np.where(by > 0, (phi - np.roll(phi, 1, axis=1)) / dom.dy, 0.0)
    gw = np.zeros((phi.shape[0] + 1,) + phi.shape[1:])
    gw[1:-1] = np.where(bz[1:] > 0, (phi[1:] - phi[:-1]) / dom.dz, 0.0)
    return gu, gv, gw


def laplacian(dom, b, phi):
    """L phi = D(G(phi))."""
    return divergence(dom, b, *gradient(dom, b, phi))


def diagonal(dom, b):
    """Diagonal of -L: sum of the face weights beta / delta^2 of each cell."""
    bx, by, bz = b
    return ((bx + np.roll(bx, -1, axis=2)) / dom.dx ** 2 + (by + np.roll(by, -1, axis=1)) / dom.dy ** 2 +
            (bz + _hi_z(bz)) / dom.dz ** 2)


def pcg(dom, b, rhs, rtol=1e-10, maxit=100000, phi0=None, atol=0.0):
    """Jacobi-preconditioned conjugate gradients on -L phi = -rhs, stopped at
    ||r|| <= max(rtol ||rhs||, atol).  The fluid above a height-function
    terrain is one connected region, so the null space of L is the constant
    field and a consistent right-hand side sums to zero over the active
    cells; its mean (rounding only) is removed first.  Returns (phi,
    iterations, relative residual)."""
    d = diagonal(dom, b)
    act = d > 0
    A = lambda x: -laplacian(dom, b, x)
    rhs = np.where(act, rhs, 0.0)
    if act.any():
        rhs = np.where(act, rhs - rhs[act].mean(), 0.0)
    bnorm = np.linalg.norm(rhs)
    phi = np.zeros_like(rhs) if phi0 is None else np.where(act, phi0, 0.0)
    if bnorm == 0.0:
        return phi, 0, 0.0
    r = -rhs - A(phi)
    r = np.where(act, r, 0.0)
    z = np.where(act, r / np.where(act, d, 1.0), 0.0)
    p = z.copy()
    rz = float(np.sum(r * z))
    it = 0
    res = np.linalg.norm(r) / bnorm
    stop = max(rtol, atol / bnorm)
    while res > stop and it < maxit:
        q = np.where(act, A(p), 0.0)
        alpha = rz / float(np.sum(p * q))
        phi = phi + alpha * p
        r = r - alpha * q
        res = np.linalg.norm(r) / bnorm
        it += 1
        if res <= stop:
            break
        z = np.where(act, r / np.where(act, d, 1.0), 0.0)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return phi, it, res


def project(dom, geom, mu, mv, mw, dt, rtol=1e-10, phi0=None, atol=0.0):
    """Projection of the face momenta onto the discretely divergence-free
    fields: returns (mu, mv, mw, phi, iterations, relative residual)."""
    b = face_weights(dom, geom)
    rhs = divergence(dom, b, mu, mv, mw) / dt
    phi, it, res = pcg(dom, b, rhs, rtol, phi0=phi0, atol=atol)
    gu, gv, gw = gradient(dom, b, phi)
    return mu - dt * gu, mv - dt * gv, mw - dt * gw, phi, it, res


def anelastic_step(oracle, dom, geom, tables, U, dt, rtol=1e-10):
    """One step of Algorithm 2 with two stages in the low-storage form
    U* = P[R[U + dt/2 dU(U)]], U' = P[R[U + dt dU(U*)]]: the flux update and
    redistribution of the compressible path with the density held at the
    reference (rho perturbation zero), then the projection P of the face
    momenta.  U holds full values; rho must equal the reference profile.
    Returns (U', iterations of each projection)."""
    its = []
    cur = {f: np.array(v, copy=True) for f, v in U.items()}
    rho0 = np.array(U["rho"], copy=True)
    for frac in (0.5, 1.0):
        dU = oracle.flux_div(dom, geom, cur)
        hat = {f: U[f] + dt * frac * dU[f] for f in U}
        nxt = {}
        for f in U:
            g = {"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}[f]
            nxt[f] = oracle.wsrd(dom, geom, tables, g, hat[f])
        nxt["rho"] = rho0.copy()
        mu, mv, mw, _, it, _ = project(dom, geom, nxt["rhou"], nxt["rhov"], nxt["rhow"], dt * frac, rtol)
        nxt["rhou"], nxt["rhov"], nxt["rhow"] = mu, mv, mw
        its.append(it)
        cur = nxt
    return cur, its
