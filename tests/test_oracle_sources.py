"""Pins of the oracle's sources of the compressible system (Sec. 2.1, Eq.
mom-comp): the perturbation pressure gradient -grad p' with p from the
equation of state p = P00 (R rho theta / P00)^gamma, and the buoyancy
B = -rho' g on rho*w.  Each pin fails on a named mutation of oracle/eb_oracle.c
(section 4), given in its docstring."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


def _case(oracle, terrain="flat", nx=24, ny=20, nz=12, **kw):
    # flat terrain at 0.25 = level 6 of 12 over Lz = 0.5: a grid-aligned floor,
    # no cut CVs
    kw.setdefault("hmax", 0.25)
    w = inputs.Workload("t", nx, ny, nz, 1, terrain=terrain, **kw)
    h = w.heights()
    dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h)
    G = oracle.geometry(dom)
    r0, rt0 = inputs.cell_reference(w.nz, w.Lz)
    return w, dom, G, np.asarray(r0), np.asarray(rt0)


def _rest(dom, r0, rt0):
    U = {f: np.zeros(dom.shape(3 if f == "rhow" else 0)) for f in FIELDS}
    U["rho"][:] = r0[:, None, None]
    U["rhotheta"][:] = rt0[:, None, None]
    return U


def _pprime(rt, rt0):
    """p - p0 of the equation of state (Sec. 2.1), evaluated at 40 digits
    from the FP64 inputs: R = 287, cp = 1004.5, gamma = cp / (cp - R),
    P00 = 1e5."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    R, P00 = mpmath.mpf(287), mpmath.mpf(100000)
    gam = mpmath.mpf("1004.5") / (mpmath.mpf("1004.5") - R)
    out = np.empty(rt.shape)
    for idx in np.ndindex(rt.shape):
        k = idx[0]
        out[idx] = float(P00 * ((R * mpmath.mpf(float(rt[idx])) / P00) ** gam
                                - (R * mpmath.mpf(float(rt0[k])) / P00) ** gam))
    return out


def test_equation_of_state_closed_forms(oracle):
    """p = P00 where R rho theta = P00, whatever gamma; multiplying rho theta
    by 2^(1/gamma) with gamma = cp / (cp - R) = 1.4 doubles p.  Fails if P00,
    R or gamma (cp) is wrong, or if the exponent is applied to p instead of
    R rho theta / P00."""
    R, P00 = 287.0, 1.0e5
    assert oracle.eos_pressure(P00 / R) == pytest.approx(P00, rel=1e-14)
    for x in (250.0, 348.4, 401.0):
        assert oracle.eos_pressure(x * 2.0 ** (1.0 / 1.4)) / oracle.eos_pressure(x) == pytest.approx(2.0, rel=1e-13)
    assert oracle.eos_pressure(2.0 * P00 / R) == pytest.approx(P00 * 2.0 ** 1.4, rel=1e-14)


def test_rest_state_stays_at_rest(oracle):
    """The reference state at rest over a grid-aligned floor is an exact
    steady state of the step with both sources (forward Euler and the
    three-stage form): p' = 0 and rho' = 0 everywhere.  Fails if the full
    pressure p (or its hydrostatic part) is differentiated instead of p', or
    if the buoyancy takes rho instead of rho'."""
    w, dom, G, r0, rt0 = _case(oracle)
    T = oracle.wsrd_setup(dom, G)
    U = _rest(dom, r0, rt0)
    S = oracle.Sources(r0, rt0)
    dt = 0.3 * dom.dz / 350.0
    for stages, n in ((1, 3), (3, 1)):
        V = oracle.step(dom, G, T, U, dt, n, stages, S)
        for f in FIELDS:
            assert np.array_equal(V[f], U[f]), (stages, f)


def test_pressure_gradient_closed_form(oracle):
    """Zero momenta, rho = rho0 and a rho*theta perturbation varying in x, y
    and z: the source of every momentum CV with two fluid cells is
    -(p'_b - p'_a) / dx_d, a the cell one step back along its staggering axis,
    b the cell of the same index; the c grid gets none, and the w CV on the
    floor (its lower cell covered) none.  Fails on a sign flip, on the
    forward instead of the backward cell (i + 1 for i - 1), on dx for dy or
    dz, or on a missing 1/dx."""
    w, dom, G, r0, rt0 = _case(oracle)
    U = _rest(dom, r0, rt0)
    z = (np.arange(dom.nz) + 0.5) * dom.dz
    y = (np.arange(dom.NY) + 0.5) * dom.dy
    x = (np.arange(dom.NX) + 0.5) * dom.dx
    f = (np.sin(2 * np.pi * x / w.Lx)[None, None, :] + 0.5 * np.cos(2 * np.pi * y / w.Ly)[None, :, None]
         + 2.0 * z[:, None, None])
    U["rhotheta"] = U["rhotheta"] + 0.5 * f
    S = oracle.Sources(r0, rt0, pressure=True, buoyancy=False)
    dU = oracle.sources(dom, G, U, S)
    pp = _pprime(U["rhotheta"], rt0)
    fluid = G[0]["alpha"] > 0
    kf = 6   # the first fluid level
    assert not fluid[kf - 1].any() and fluid[kf:].all()
    want_u = -(pp - np.roll(pp, 1, axis=2)) / dom.dx
    want_v = -(pp - np.roll(pp, 1, axis=1)) / dom.dy
    want_w = np.zeros_like(U["rhow"])
    want_w[kf + 1:dom.nz] = -(pp[kf + 1:] - pp[kf:-1]) / dom.dz
    scale = np.abs(want_u[kf:]).max()
    assert np.abs(dU["rhou"][kf:] - want_u[kf:]).max() <= 1e-12 * scale
    assert np.abs(dU["rhov"][kf:] - want_v[kf:]).max() <= 1e-12 * scale
    assert np.abs(dU["rhow"] - want_w).max() <= 1e-12 * scale
    assert not dU["rhou"][:kf].any() and not dU["rhov"][:kf].any()
    assert not dU["rho"].any() and not dU["rhotheta"].any()


def test_buoyancy_closed_form(oracle):
    """rho*theta = rho0 theta0 (p' = 0) and a density anomaly rho': the w CVs
    get -g (rho'_a + rho'_b) / 2 of their two cells, the floor CV -g rho'_b
    (its lower cell covered), the u and v CVs nothing.  Fails on a sign flip,
    on g other than 9.81, on one cell's rho' instead of the mean, or on the
    buoyancy landing on rho*u or rho*v."""
    w, dom, G, r0, rt0 = _case(oracle)
    U = _rest(dom, r0, rt0)
    rng = np.random.default_rng(4)
    rp = 1e-3 * rng.standard_normal(U["rho"].shape)
    U["rho"] = U["rho"] + rp
    S = oracle.Sources(r0, rt0, pressure=False, buoyancy=True)
    dU = oracle.sources(dom, G, U, S)
    kf = 6
    want = np.zeros_like(U["rhow"])
    want[kf + 1:dom.nz] = -9.81 * 0.5 * (rp[kf:-1] + rp[kf + 1:])
    want[kf] = -9.81 * rp[kf]
    assert np.abs(dU["rhow"] - want).max() <= 1e-12 * np.abs(want).max()
    for f in ("rho", "rhotheta", "rhou", "rhov"):
        assert not dU[f].any(), f


def test_no_pressure_force_across_a_wall_side(oracle):
    """On a hill, a u CV whose low or high cell is covered gets no pressure
    source (the covered cell takes the fluid cell's p'), while every u CV
    with two fluid cells gets the closed form.  Fails if the covered cell's
    own (stored) value is used, or if such CVs are skipped altogether (the
    closed form then fails on the CVs next to them)."""
    w, dom, G, r0, rt0 = _case(oracle, terrain="gaussian", nx=32, ny=24, nz=16, hmax=0.3)
    U = _rest(dom, r0, rt0)
    x = (np.arange(dom.NX) + 0.5) * dom.dx
    U["rhotheta"] = U["rhotheta"] + 0.8 * np.sin(2 * np.pi * x / w.Lx)[None, None, :]
    U["rhotheta"][G[0]["alpha"] == 0] = 123.0    # stored values in covered cells must not matter
    S = oracle.Sources(r0, rt0, pressure=True, buoyancy=False)
    dU = oracle.sources(dom, G, U, S)
    fc = G[0]["alpha"] > 0
    fu = G[1]["alpha"] > 0
    fa = np.roll(fc, 1, axis=2)
    one_side = fu & (fa != fc)
    both = fu & fa & fc
    assert one_side.sum() > 0
    assert not dU["rhou"][one_side].any()
    pp = _pprime(U["rhotheta"], rt0)
    want = -(pp - np.roll(pp, 1, axis=2)) / dom.dx
    assert np.abs(dU["rhou"][both] - want[both]).max() <= 1e-12 * np.abs(want[both]).max()
