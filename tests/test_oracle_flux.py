"""Pins of the oracle's fluxes, cut-cell update and step (Sec. 3.1, 4.1,
Algorithm 1 with S = 0): exactness of the upwind interpolant on cubics, flux
closure at cut cells, centroid interpolation of a linear flux, conservation,
a grid-aligned terrain against the scheme without EB, symmetry, and the
stabilising effect of redistribution.  CPU only."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs


def flat_domain(oracle, nx, ny, nz, H=0.0, L=(1.0, 1.0, 0.5)):
    dz = L[2] / nz
    h = np.full((ny + 1, nx + 1), H * dz)
    dom = oracle.Domain(nx, ny, nz, L[0], L[1], L[2], h)
    return dom, oracle.geometry(dom)


def const_state(dom, rho=1.0, rt=1.0, ru=0.0, rv=0.0, rw=0.0):
    U = {n: np.zeros(dom.shape(g)) for n, g in (("rho", 0), ("rhotheta", 0), ("rhou", 1), ("rhov", 2),
                                              ("rhow", 3))}
    U["rho"][:] = rho
    U["rhotheta"][:] = rt
    U["rhou"][:] = ru
    U["rhov"][:] = rv
    U["rhow"][1:dom.nz] = rw
    return U


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_upwind_exact_on_cubics(oracle, axis, sign):
    """With a uniform mass flux m, the third-order upwind flux difference is
    exact for cubic profiles: d(rho theta) = -m theta'(x) at cell centres
    (Sec. 4.1, fourth-order centred plus hyperviscosity)."""
    n = 24
    dom, G = flat_domain(oracle, n, n, n, L=(1.0, 1.0, 1.0))
    vel = [0.0, 0.0, 0.0]
    vel[axis] = sign
    U = const_state(dom, ru=vel[0], rv=vel[1], rw=vel[2])
    c = (np.arange(n) + 0.5) / n
    th = 1.0 + 0.3 * c - 0.8 * c ** 2 + 0.5 * c ** 3
    dth = (0.3 - 1.6 * c + 1.5 * c ** 2)
    shp = [1, 1, 1]
    shp[2 - axis] = n
    U["rhotheta"] = np.ascontiguousarray(np.broadcast_to(th.reshape(shp), dom.shape(0)))
    dU = oracle.flux_div(dom, G, U)
    got = np.moveaxis(dU["rhotheta"], 2 - axis, 0)
    want = -sign * dth[:, None, None]
    assert np.max(np.abs(got[3:n - 3] - want[3:n - 3])) < 1e-11
    # mass is uniform: no density change away from walls / periodic seams
    assert np.max(np.abs(np.moveaxis(dU["rho"], 2 - axis, 0)[3:n - 3])) < 1e-12


@pytest.mark.parametrize("case", ["u_by_v", "v_by_w", "w_by_u"])
def test_momentum_grids_upwind_exact(oracle, case):
    """Each face grid advects its velocity with the mass flux of the edge
    faces: u along y by rho v, v along z by rho w, w along x by rho u; a cubic
    velocity profile gives d(rho u_a) = -u_a'(x_b) exactly."""
    n = 24
    dom, G = flat_domain(oracle, n, n, n, L=(1.0, 1.0, 1.0))
    U = const_state(dom)
    e = np.arange(n) / n                 # edge positions of the faces along the advection axis
    cc = (np.arange(n) + 0.5) / n        # cell-centre positions
    prof = lambda x: 0.2 + 0.4 * x - 0.9 * x ** 2 + 0.6 * x ** 3
    dprof = lambda x: 0.4 - 1.8 * x + 1.8 * x ** 2
    if case == "u_by_v":
        U["rhov"][:] = 1.0
        U["rhou"][:] = prof(cc)[None, :, None]
        got, want, lo = dU_of(oracle, dom, G, U, "rhou")[:, :, :], -dprof(cc)[None, :, None], (slice(None), slice(3, n - 3), slice(None))
    elif case == "v_by_w":
        U["rhow"][1:n] = -1.0
        U["rhov"][:] = prof(cc)[:, None, None]
        got, want, lo = dU_of(oracle, dom, G, U, "rhov"), dprof(cc)[:, None, None], (slice(3, n - 3), slice(None), slice(None))
    else:
        U["rhou"][:] = 1.0
        U["rhow"][1:n] = prof(cc)[None, None, :]
        got, want, lo = dU_of(oracle, dom, G, U, "rhow"), -dprof(cc)[None, None, :], (slice(3, n - 3), slice(None), slice(3, n - 3))
    g = got[lo]
    w = np.broadcast_to(want, got.shape)[lo]
    assert np.max(np.abs(g - w)) < 1e-11


def dU_of(oracle, dom, G, U, f):
    return oracle.flux_div(dom, G, U)[f]


@pytest.fixture(scope="module")
def ridge(oracle):
    w = inputs.WOA_32
    dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, w.heights())
    G = oracle.geometry(dom)
    return w, dom, G, oracle.wsrd_setup(dom, G)


def test_cut_cell_flux_closure(ridge, oracle):
    """Uniform mass flux m = 1 along x and zero EB flux: every open face
    carries exactly m, so a cut cell gains -(beta_hi - beta_lo) m / (alpha dx),
    which by the discrete divergence theorem is -ebv_x m / (alpha dx)."""
    w, dom, G, T = ridge
    U = const_state(dom, ru=1.0)
    dU = oracle.flux_div(dom, G, U)
    cut = (G[0]["flag"] == 2) & (G[0]["alpha"] > 0)
    want = np.zeros_like(dU["rho"])
    want[cut] = -G[0]["ebv"][0][cut] / (G[0]["alpha"][cut] * dom.dx)
    assert cut.sum() > 100
    assert np.allclose(dU["rho"][cut], want[cut], rtol=1e-12, atol=1e-9)
    reg = G[0]["flag"] == 1
    assert np.all(dU["rho"][reg] == 0.0)


def test_centroid_interpolation_linear_flux(ridge, oracle):
    """rho u = a + b z: the provisional mass flux is linear in z, so the
    bilinear interpolation toward the face centroid returns its value at the
    centroid height (Sec. 4.1).  On the y-uniform ridge every x-face centroid
    lies above the face centre, where the neighbour face is open."""
    w, dom, G, T = ridge
    a, b = 0.7, 1.9
    U = const_state(dom)
    zc = (np.arange(dom.nz) + 0.5) * dom.dz
    U["rhou"][:] = (a + b * zc)[:, None, None]
    dU = oracle.flux_div(dom, G, U)
    beta, gz = G[0]["beta"][0], G[0]["fcent"][1]
    F = a + b * (zc[:, None, None] + gz * dom.dz)
    Fhi = np.roll(beta * F, -1, axis=2)
    act = G[0]["alpha"] > 0
    want = np.zeros_like(F)
    want[act] = -(Fhi - beta * F)[act] / (G[0]["alpha"][act] * dom.dx)
    k_ok = np.zeros_like(act)
    k_ok[: dom.nz - 1] = True
    sel = act & k_ok
    assert np.any(gz[sel] > 0.05)
    assert np.allclose(dU["rho"][sel], want[sel], rtol=1e-12, atol=1e-10)


def test_flux_divergence_conservative(oracle):
    """sum alpha dU = 0 for every field of a random state on rough terrain
    (telescoping flux form, zero EB flux); for rho w the wall-adjacent w levels
    are set to zero so that no flux crosses into the non-prognostic walls."""
    nx, ny, nz = 20, 18, 12
    h = inputs.grf_terrain(nx, ny, seed=9, hmax=0.2)
    dom = oracle.Domain(nx, ny, nz, 1.0, 1.0, 0.5, h)
    G = oracle.geometry(dom)
    U = inputs.initial_state(nx, ny, nz, 0.5, pert=0.05, seed=2)
    U["rhow"][1] = 0.0
    U["rhow"][nz - 1] = 0.0
    dU = oracle.flux_div(dom, G, U)
    for f, g in (("rho", 0), ("rhotheta", 0), ("rhou", 1), ("rhov", 2), ("rhow", 3)):
        s = (G[g]["alpha"] * dU[f]).sum()
        scale = (G[g]["alpha"] * np.abs(dU[f])).sum()
        assert abs(s) <= 1e-13 * scale, f


@pytest.mark.parametrize("stages", [1, 3])
def test_step_conservation(oracle, stages):
    """Whole steps conserve sum alpha U on every grid to round-off."""
    nx, ny, nz = 16, 16, 12
    h = inputs.gaussian_hill(nx, ny, h0=0.2, sigma=0.12)
    dom = oracle.Domain(nx, ny, nz, 1.0, 1.0, 0.5, h)
    G = oracle.geometry(dom)
    T = oracle.wsrd_setup(dom, G)
    U0 = inputs.initial_state(nx, ny, nz, 0.5, pert=0.01, seed=7)
    U0["rhow"][1] = 0.0
    U0["rhow"][nz - 1] = 0.0
    U1 = oracle.step(dom, G, T, U0, inputs.fixed_dt(nx, ny, nz, 1, 1, 0.5), 1, stages)
    for f, g in (("rho", 0), ("rhotheta", 0), ("rhou", 1), ("rhov", 2)):
        a = (G[g]["alpha"] * U0[f]).sum()
        b = (G[g]["alpha"] * U1[f]).sum()
        sc = (G[g]["alpha"] * np.abs(U0[f])).sum()
        assert abs(a - b) <= 1e-13 * sc, f
    if stages == 1:
        act = G[3]["alpha"].copy()
        act[0] = act[nz] = 0.0
        assert abs((act * U0["rhow"]).sum() - (act * U1["rhow"]).sum()) <= 1e-13 * (act * np.abs(U0["rhow"])).sum()


@pytest.mark.parametrize("m", [2, 3])
def test_grid_aligned_terrain_matches_no_eb(oracle, m):
    """Terrain exactly on the plane z = m dz with w = 0 initially reproduces the
    scheme without EB on [m dz, Lz] bit for bit (the wall w face keeps w = 0;
    it is updated by the EB scheme, Sec. 3.2, but its update is zero)."""
    nx, ny, nz = 12, 10, 8
    dz = 0.5 / nz            # 1/16: the terrain plane and the reduced domain are exact
    domA, GA = flat_domain(oracle, nx, ny, nz, H=m)
    TA = oracle.wsrd_setup(domA, GA)
    Lz_b = 0.5 - m * dz
    domB, GB = flat_domain(oracle, nx, ny, nz - m, H=0.0, L=(1.0, 1.0, Lz_b))
    TB = oracle.wsrd_setup(domB, GB)
    assert domB.dz == dz
    rng = np.random.default_rng(1)
    UA = inputs.initial_state(nx, ny, nz, 0.5, u0=(1.0, 0.6, 0.0), pert=0.02, seed=3)
    UA["rhow"][:] = 0.0
    UB = {f: np.ascontiguousarray(v[m:]) for f, v in UA.items()}
    dt = inputs.fixed_dt(nx, ny, nz, 1, 1, 0.5, u0=(1.0, 0.6, 0.0))
    RA = oracle.step(domA, GA, TA, UA, dt, 3)
    RB = oracle.step(domB, GB, TB, UB, dt, 3)
    for f in ("rho", "rhotheta", "rhou", "rhov"):
        assert np.array_equal(RA[f][m:], RB[f]), f
    assert np.array_equal(RA["rhow"][m + 1:], RB["rhow"][1:])
    assert np.all(RA["rhow"][m] == 0.0)


def test_ridge_symmetry(ridge, oracle):
    """The y-uniform ridge with a y-uniform state stays y-uniform bit for bit,
    and rho v stays zero."""
    w, dom, G, T = ridge
    U = w.state("uniform")
    R = oracle.step(dom, G, T, U, w.dt(), w.steps)
    for f, a in R.items():
        assert np.array_equal(a, np.broadcast_to(a[:, :1, :], a.shape)), f
    assert np.all(R["rhov"] == 0.0)
    assert np.all(np.isfinite(R["rho"]))


def test_redistribution_stabilises_small_cells(ridge, oracle):
    """Five steps with and without redistribution (V_target -> 0 removes every
    merging neighbourhood): without it the small cut cells take updates of
    order dt / alpha (Sec. 6.1 shows nonphysical values), with it they stay
    near their neighbours."""
    w, dom, G, T = ridge
    T0 = oracle.wsrd_setup(dom, G, vt=1e-300)
    assert all((T0[g]["code"] > 0).sum() == 0 for g in range(4))
    U = w.state("uniform")
    on = oracle.step(dom, G, T, U, w.dt(), 5)
    off = oracle.step(dom, G, T0, U, w.dt(), 5)
    small = (T[0]["code"] > 0)
    dev_on = np.max(np.abs(on["rho"][small] - U["rho"][small]) / U["rho"][small])
    dev_off = np.max(np.abs(off["rho"][small] - U["rho"][small]) / U["rho"][small])
    assert dev_off > 5 * dev_on
