"""Ensembles (eb_ensemble_*): members of uneven sizes advanced together by
graph replay must give exactly what eb_step gives for each member alone
(same kernels, same arithmetic; the work split and the tuned slab heights
change only who computes what), in both precisions."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import FIELDS, make_geometry, refs_for, to_device

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11959_gb300 import eb as _eb
    _eb.load(build_if_missing=True)
    return _eb


def members():
    return [
        inputs.Workload("hill-32x32x16", 32, 32, 16, 1, terrain="gaussian", hmax=0.12),
        inputs.Workload("grf-48x40x24", 48, 40, 24, 1, terrain="grf", seed=5, hmax=0.2, tiny=3),
        inputs.Workload("woa-64x32x20", 64, 32, 20, 1, terrain="woa", hmax=0.1),
        inputs.Workload("grf-45x38x20", 45, 38, 20, 1, terrain="grf", seed=9, hmax=0.2, tiny=2),
        inputs.Workload("hill-96x64x40", 96, 64, 40, 1, terrain="gaussian", hmax=0.2),
    ]


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_ensemble_equals_each_member_alone(eb, precision):
    ws = members()
    geoms, states, dts, refs = [], [], [], []
    for q, w in enumerate(ws):
        r = refs_for(w.nz, w.Lz)
        refs.append(r)
        geoms.append(make_geometry(eb, w, w.heights(), precision, r))
        states.append(to_device(w.state("sheltered", seed=q), precision, r))
        dts.append(w.dt())
    nsteps = 3
    want = [eb.step(g, U, dt, nsteps) for g, U, dt in zip(geoms, states, dts)]
    ens = eb.Ensemble(geoms)
    for q, U in enumerate(states):
        ens.set_state(q, U)
    ens.step(dts, nsteps)
    for q in range(len(ws)):
        got = ens.get_state(q)
        for f in FIELDS:
            assert torch.equal(got[f], want[q][f]), (precision, ws[q].name, f)
    # tuned slab heights: the same results again from the same states
    best = ens.tune(dts, reps=1)
    assert best in (0, 8, 16, 24, 32, 48, 64) or best >= 64
    for q, U in enumerate(states):
        ens.set_state(q, U)
    ens.step(dts, 1)
    ens.step(dts, nsteps - 1)
    for q in range(len(ws)):
        got = ens.get_state(q)
        for f in FIELDS:
            assert torch.equal(got[f], want[q][f]), ("tuned", precision, ws[q].name, f)
    for g in geoms:
        eb.sync_status(g)
    ens.close()


def test_tuning_leaves_the_loaded_states(eb):
    ws = members()[:2]
    geoms = [make_geometry(eb, w, w.heights(), "mixed", refs_for(w.nz, w.Lz)) for w in ws]
    states = [to_device(w.state("sheltered", seed=7), "mixed", refs_for(w.nz, w.Lz)) for w in ws]
    ens = eb.Ensemble(geoms)
    for q, U in enumerate(states):
        ens.set_state(q, U)
    ens.tune([w.dt() for w in ws], reps=1)
    for q in range(len(ws)):
        got = ens.get_state(q)
        for f in FIELDS:
            assert torch.equal(got[f], states[q][f])
    ens.close()


def test_ensemble_argument_errors(eb):
    w = members()[0]
    r = refs_for(w.nz, w.Lz)
    g64 = make_geometry(eb, w, w.heights(), "f64", r)
    g32 = make_geometry(eb, w, w.heights(), "mixed", r)
    with pytest.raises(eb.EbError):
        eb.Ensemble([])
    with pytest.raises(eb.EbError):
        eb.Ensemble([g64, g32])
    with pytest.raises(eb.EbError):
        eb.Ensemble([g64, g64])
    ens = eb.Ensemble([g64])
    with pytest.raises(eb.EbError):
        ens.step([-1.0], 1)
    with pytest.raises(ValueError):
        ens.step([1e-3, 1e-3], 1)
    ens.close()
