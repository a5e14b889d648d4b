"""The sources of the compressible system (Sec. 2.1, Eq. mom-comp) in eb_step
(eb_geom_set_sources) against the oracle: the perturbation pressure gradient
from the equation of state and the buoyancy, added to the flux divergence of
every stage before the redistribution.  A hill and a rough random terrain
with planted tiny cells, the sheltered state with its background wind, a
time step that resolves sound waves; forward Euler and the three-stage form,
both precisions, to the tolerances of the advection-only steps (FP64 1e-12,
mixed 1e-5).  The FP64 momenta are measured on the scale of the largest
momentum component: with the pressure source the oracle's own full-value
state limits it there (one ulp of rho*theta ~ 350 moves p' by 2e-11 Pa; a
random one-ulp change of the oracle's input moves rho*v and rho*w by up to
8e-13 of their own largest values after two three-stage steps, against 4e-16
without the sources), while the FP64 path stores perturbations."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import FGRID, FIELDS, TOL, active_masks, make_geometry, rel_linf, to_device, to_host, wind_refs, worst

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "hill": inputs.Workload("hill-48x40x24", 48, 40, 24, 4, terrain="gaussian", hmax=0.15),
    "grf": inputs.Workload("grf-48x40x24", 48, 40, 24, 4, terrain="grf", seed=5, hmax=0.2, tiny=3),
}


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11959_gb300 import build, eb as ebmod
    build.build()
    ebmod.load()
    return ebmod


def acoustic_dt(w):
    """A time step at which sound (about 350 m/s) crosses 0.3 of a cell."""
    return 0.3 * min(w.Lx / w.nx, w.Ly / w.ny, w.Lz / w.nz) / (1.0 + 350.0)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, oracle):
    w = CASES[request.param]
    h = w.heights()
    dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h)
    G = oracle.geometry(dom)
    T = oracle.wsrd_setup(dom, G)
    return request.param, w, h, dom, G, T


@pytest.mark.parametrize("precision,stages", [("f64", 1), ("mixed", 1), ("f64", 3), ("mixed", 3)])
def test_steps_with_sources_match(eb, case, oracle, precision, stages):
    name, w, h, dom, G, T = case
    refs = wind_refs(w, "sheltered")
    U = w.state("sheltered", seed=8)
    dt = acoustic_dt(w)
    nsteps = 4 if stages == 1 else 2
    src = oracle.Sources(refs[0], refs[1], pressure=True, buoyancy=True)
    want = oracle.step(dom, G, T, U, dt, nsteps, stages, src)
    plain = oracle.step(dom, G, T, U, dt, nsteps, stages)
    geom = make_geometry(eb, w, h, precision, refs)
    geom.set_sources(pressure=True, buoyancy=True)
    got = to_host(eb.step(geom, to_device(U, precision, refs), dt, nsteps, stages), refs)
    eb.sync_status(geom)
    geom.close()
    act = active_masks(G, w.nz)
    mom = max(float(np.abs(want[f][act[FGRID[f]]]).max()) for f in ("rhou", "rhov", "rhow"))
    for f in FIELDS:
        g = FGRID[f]
        d = float(np.abs(got[f] - want[f])[act[g]].max())
        own = float(np.abs(want[f][act[g]]).max())
        err = d / (mom if precision == "f64" and g else own)
        assert err <= TOL[precision], (name, precision, stages, f, err, d / own, worst(got[f], want[f], act[g]))
    # the sources matter: the momenta move well beyond the tolerance
    for f in ("rhou", "rhov", "rhow"):
        assert rel_linf(plain[f], want[f], act[FGRID[f]]) > 100 * TOL["mixed"], f


@pytest.mark.parametrize("flags", [(True, False), (False, True)])
def test_each_source_alone(eb, case, oracle, flags):
    """The pressure gradient and the buoyancy switched on one at a time
    (FP64 path, two forward-Euler steps)."""
    name, w, h, dom, G, T = case
    refs = wind_refs(w, "sheltered")
    U = w.state("sheltered", seed=9)
    dt = acoustic_dt(w)
    want = oracle.step(dom, G, T, U, dt, 2, 1, oracle.Sources(refs[0], refs[1], *flags))
    geom = make_geometry(eb, w, h, "f64", refs)
    geom.set_sources(*flags)
    got = to_host(eb.step(geom, to_device(U, "f64", refs), dt, 2, 1), refs)
    eb.sync_status(geom)
    geom.close()
    act = active_masks(G, w.nz)
    mom = max(float(np.abs(want[f][act[FGRID[f]]]).max()) for f in ("rhou", "rhov", "rhow"))
    for f in FIELDS:
        g = FGRID[f]
        d = float(np.abs(got[f] - want[f])[act[g]].max())
        err = d / (mom if g else float(np.abs(want[f][act[g]]).max()))
        assert err <= TOL["f64"], (name, flags, f, err)


def test_sources_off_is_the_plain_step(eb):
    """Switching the sources on and off again gives the plain step bit for
    bit; a handle without reference profiles refuses them, and so do the
    ensembles and unknown flag bits."""
    w = CASES["hill"]
    h = w.heights()
    refs = wind_refs(w, "sheltered")
    U = w.state("sheltered", seed=10)
    geom = make_geometry(eb, w, h, "mixed", refs)
    A = to_device(U, "mixed", refs)
    want = eb.step(geom, A, w.dt(), 2)
    geom.set_sources(True, True)
    moved = eb.step(geom, A, acoustic_dt(w), 1)
    geom.set_sources(False, False)
    got = eb.step(geom, A, w.dt(), 2)
    for f in FIELDS:
        assert torch.equal(got[f], want[f]), f
        assert torch.isfinite(moved[f]).all(), f
    geom.set_sources(True, False)
    with pytest.raises(eb.EbError) as e:
        eb.Ensemble([geom])
    assert e.value.code == 6
    with pytest.raises(eb.EbError) as e:
        eb._check(eb.load().eb_geom_set_sources(geom.handle, 4))
    assert e.value.code == 1
    geom.set_sources(False, False)
    eb.sync_status(geom)
    geom.close()
    bare = make_geometry(eb, w, h, "mixed", None)
    with pytest.raises(eb.EbError) as e:
        bare.set_sources(True, True)
    assert e.value.code == 6
    bare.close()
