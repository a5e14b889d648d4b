"""The projection with the multigrid preconditioner (EB_PRECOND_MG): the same
projection as the FP64 oracle's Jacobi-preconditioned conjugate gradients
(the preconditioner changes the path to the solution, not the solution), in
far fewer iterations; deterministic; rejected on grids it cannot coarsen."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import make_geometry, refs_for

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


def _state(w, m, dtype):
    shape = (w.nz, w.ny, w.nx)
    return {"rho": torch.zeros(shape, dtype=dtype, device="cuda"),
            "rhotheta": torch.zeros(shape, dtype=dtype, device="cuda"),
            **{f: torch.from_numpy(m[f]).to(device="cuda", dtype=dtype) for f in m}}


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_mg_projection_matches_oracle(eb, proj, case, precision):
    name, w, h, dom, geom = case
    m = _momenta(dom, geom, 21)
    dt = 0.5 * w.Lx / w.nx
    dtype = torch.float64 if precision == "f64" else torch.float32
    U = _state(w, m, dtype)
    host = {f: U[f].double().cpu().numpy() for f in m}
    geo = make_geometry(eb, w, h, precision, refs_for(w.nz, w.Lz))
    eb.set_preconditioner(geo, "mg")
    it, res = eb.project(geo, U, dt, rtol=1e-12)
    mu, mv, mw, _, it_o, res_o = proj.project(dom, geom, host["rhou"], host["rhov"], host["rhow"], dt, rtol=1e-12)
    assert res <= 1e-12 and res_o <= 1e-12
    assert it * 4 <= it_o, (name, it, it_o)   # multigrid: far fewer iterations than Jacobi
    scale = max(np.max(np.abs(x)) for x in (mu, mv, mw))
    for f, want in (("rhou", mu), ("rhov", mv), ("rhow", mw)):
        err = np.max(np.abs(U[f].double().cpu().numpy() - want)) / scale
        assert err <= TOL[precision], (name, precision, f, err)
    geo.close()


def test_mg_and_jacobi_give_the_same_anelastic_step(eb, case):
    name, w, h, dom, geom = case
    refs = refs_for(w.nz, w.Lz)
    U0 = w.state("sheltered", seed=3)
    U0 = {f: np.array(v, copy=True) for f, v in U0.items()}
    U0["rho"] = np.broadcast_to(refs[0][:, None, None], U0["rho"].shape).copy()
    outs, its = [], []
    for kind in ("jacobi", "mg"):
        geo = make_geometry(eb, w, h, "f64", refs)
        eb.set_preconditioner(geo, kind)
        A = eb.device_state(U0, "f64", refs)
        out, it = eb.anelastic_step(geo, A, w.dt(), 1, rtol=1e-12)
        outs.append({f: out[f].clone() for f in out})
        its.append(sum(it))
        geo.close()
    assert its[1] * 4 <= its[0], (name, its)
    scale = max(float(outs[0][f].abs().max()) for f in ("rhou", "rhov", "rhow"))
    for f in ("rhou", "rhov", "rhow"):
        assert float((outs[0][f] - outs[1][f]).abs().max()) <= 1e-9 * scale, (name, f)
    ref = float(outs[0]["rhotheta"].abs().max())
    assert float((outs[0]["rhotheta"] - outs[1]["rhotheta"]).abs().max()) <= 1e-9 * max(ref, scale)


def test_mg_projection_is_deterministic(eb, case):
    name, w, h, dom, geom = case
    m = _momenta(dom, geom, 5)
    geo = make_geometry(eb, w, h, "f64", refs_for(w.nz, w.Lz))
    eb.set_preconditioner(geo, "mg")
    outs = []
    for _ in range(2):
        U = _state(w, m, torch.float64)
        it, _ = eb.project(geo, U, 0.01, rtol=1e-10)
        outs.append((it, U))
    assert outs[0][0] == outs[1][0]
    for f in ("rhou", "rhov", "rhow"):
        assert torch.equal(outs[0][1][f], outs[1][1][f])
    geo.close()


def test_mg_needs_a_grid_it_can_coarsen(eb):
    w = inputs.Workload("grf-45x38x20", 45, 38, 20, 1, terrain="grf", seed=9, hmax=0.2)
    geo = make_geometry(eb, w, w.heights(), "f64", refs_for(w.nz, w.Lz))
    with pytest.raises(RuntimeError, match="coarsen"):
        eb.set_preconditioner(geo, "mg")
    with pytest.raises(ValueError):
        eb.set_preconditioner(geo, "ilu")
    eb.set_preconditioner(geo, "jacobi")
    geo.close()
