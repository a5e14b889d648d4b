"""Parity of the CUDA projection (eb_project) and anelastic step
(eb_anelastic_step) with the FP64 oracle (oracle/eb_project.py).  Both sides
solve to a relative residual of 1e-12, so the corrected momenta agree to
the solve's accuracy: 1e-9 relative (double path) or float rounding (mixed
path)."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import FIELDS, make_geometry, refs_for, rel_linf, to_device, to_host

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-9, "mixed": 2e-6}


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11959_gb300 import eb as _eb
    _eb.load(build_if_missing=True)
    return _eb


@pytest.fixture(scope="module")
def proj():
    from oracle import eb_project
    return eb_project


CASES = {
    "grf": inputs.Workload("grf-48x40x24", 48, 40, 24, 1, terrain="grf", seed=5, hmax=0.2, tiny=3),
    "hill": inputs.Workload("hill-64x64x32", 64, 64, 32, 1, terrain="gaussian", hmax=0.15),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, oracle):
    w = CASES[request.param]
    h = w.heights()
    dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h)
    return request.param, w, h, dom, oracle.geometry(dom)


def _momenta(dom, geom, seed):
    rng = np.random.default_rng(seed)
    m = {}
    for g, f in ((1, "rhou"), (2, "rhov"), (3, "rhow")):
        a = 1.0 + 0.5 * rng.standard_normal(dom.shape(g))
        a[geom[g]["alpha"] == 0] = 0.0
        if g == 3:
            a[0] = a[-1] = 0.0
        m[f] = a
    return m


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_projection_matches_oracle(eb, proj, case, precision):
    name, w, h, dom, geom = case
    m = _momenta(dom, geom, 21)
    dt = 0.5 * w.Lx / w.nx
    dtype = torch.float64 if precision == "f64" else torch.float32
    # both sides start from the same (rounded) momenta
    dev = {f: torch.from_numpy(m[f]).to(device="cuda", dtype=dtype) for f in m}
    host = {f: dev[f].double().cpu().numpy() for f in m}
    nz, ny, nx = w.nz, w.ny, w.nx
    U = {"rho": torch.zeros((nz, ny, nx), dtype=dtype, device="cuda"),
         "rhotheta": torch.zeros((nz, ny, nx), dtype=dtype, device="cuda"), **dev}
    geo = make_geometry(eb, w, h, precision, refs_for(w.nz, w.Lz))
    phi = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
    it, res = eb.project(geo, U, dt, rtol=1e-12, phi=phi)
    mu, mv, mw, _, it_o, res_o = proj.project(dom, geom, host["rhou"], host["rhov"], host["rhow"], dt, rtol=1e-12)
    assert res <= 1e-12 and res_o <= 1e-12
    assert abs(it - it_o) <= max(3, it_o // 20), (it, it_o)
    scale = max(np.max(np.abs(x)) for x in (mu, mv, mw))
    for f, want in (("rhou", mu), ("rhov", mv), ("rhow", mw)):
        got = U[f].double().cpu().numpy()
        err = np.max(np.abs(got - want)) / scale
        assert err <= TOL[precision], (name, precision, f, err)
    # the result is divergence-free by the oracle's own divergence
    b = proj.face_weights(dom, geom)
    d0 = np.linalg.norm(proj.divergence(dom, b, host["rhou"], host["rhov"], host["rhow"]))
    d1 = np.linalg.norm(proj.divergence(dom, b, *(U[f].double().cpu().numpy() for f in ("rhou", "rhov", "rhow"))))
    assert d1 <= (1e-10 if precision == "f64" else 1e-5) * d0
    # warm start from the solution: nothing left to do
    U2 = {"rho": U["rho"], "rhotheta": U["rhotheta"], **{f: torch.from_numpy(m[f]).to(device="cuda", dtype=dtype)
                                                         for f in m}}
    it0, res0 = eb.project(geo, U2, dt, rtol=1e-10, phi0=phi)
    assert it0 == 0 and res0 <= 1e-10
    geo.close()


def test_projection_is_deterministic(eb, case):
    name, w, h, dom, geom = case
    m = _momenta(dom, geom, 5)
    geo = make_geometry(eb, w, h, "f64", refs_for(w.nz, w.Lz))
    outs = []
    for _ in range(2):
        U = {"rho": torch.zeros(geo.shape(0), dtype=torch.float64, device="cuda"),
             "rhotheta": torch.zeros(geo.shape(0), dtype=torch.float64, device="cuda"),
             **{f: torch.from_numpy(m[f]).cuda() for f in m}}
        it, _ = eb.project(geo, U, 0.01, rtol=1e-10)
        outs.append((it, U))
    assert outs[0][0] == outs[1][0]
    for f in ("rhou", "rhov", "rhow"):
        assert torch.equal(outs[0][1][f], outs[1][1][f])
    geo.close()


def _anelastic_state(w, refs):
    U = w.state("sheltered", seed=3)
    U = {f: np.array(v, copy=True) for f, v in U.items()}
    U["rho"] = np.broadcast_to(refs[0][:, None, None], U["rho"].shape).copy()
    return U


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_anelastic_step_matches_oracle(eb, proj, oracle, precision):
    w = inputs.Workload("grf-40x32x20", 40, 32, 20, 1, terrain="grf", seed=13, hmax=0.15, tiny=2)
    h = w.heights()
    refs = refs_for(w.nz, w.Lz)
    dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h)
    G = oracle.geometry(dom)
    T = oracle.wsrd_setup(dom, G)
    U = _anelastic_state(w, refs)
    dev = to_device(U, precision, refs)
    U0 = to_host(dev, refs)   # the oracle starts from the same rounded state
    dt = w.dt()
    geo = make_geometry(eb, w, h, precision, refs)
    out, its = eb.anelastic_step(geo, dev, dt, nsteps=2, rtol=1e-12)
    eb.sync_status(geo)
    want = U0
    its_o = []
    for _ in range(2):
        want, it = proj.anelastic_step(oracle, dom, G, T, want, dt, rtol=1e-12)
        its_o += it
    got = to_host(out, refs)
    tol = 1e-9 if precision == "f64" else 1e-5
    # the float path's momenta are compared on their common scale: rho*v and
    # rho*w are small components the projection makes from rho*u, and the
    # float rounding of rho*u reaches them through the solve
    mscale = max(np.max(np.abs(want[f])) for f in ("rhou", "rhov", "rhow"))
    for f in FIELDS:
        act = G[{"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}[f]]["alpha"] > 0
        if precision == "mixed" and f in ("rhou", "rhov", "rhow"):
            err = float(np.max(np.abs(got[f] - want[f])[act]) / mscale)
        else:
            err = rel_linf(got[f], want[f], act)
        assert err <= tol, (precision, f, err)
    assert all(i > 0 for i in its) and len(its) == 4
    geo.close()


def test_anelastic_step_needs_a_reference_profile(eb):
    w = CASES["hill"]
    geo = make_geometry(eb, w, w.heights(), "f64", None)
    U = geo.empty_state()
    with pytest.raises(eb.EbError):
        eb.anelastic_step(geo, U, 1e-3)
    geo.close()
