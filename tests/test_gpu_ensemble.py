"""Ensembles (eb_ensemble_*): members of uneven sizes advanced together by
one persistent cooperative launch per step must give exactly what eb_step
gives for each member alone (same device functions, same arithmetic; the
work split and the tuned slab heights change only who computes what), in
both precisions; a member must match the oracle; and a CTA that never
arrives at the kernel's grid barrier must end the step with EB_ERR_TIMEOUT,
not a hang."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import FGRID, FIELDS, TOL, active_masks, make_geometry, refs_for, rel_linf, to_device, to_host

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


@pytest.mark.parametrize("schedule", ["persistent", "branches"])
@pytest.mark.parametrize("precision,ragged", [("f64", True), ("mixed", True), ("mixed", False)])
def test_ensemble_equals_each_member_alone(eb, precision, ragged, schedule):
    """ragged: a member whose rows do not suit 16-byte copies makes the whole
    ensemble use the element-wise variant of the persistent kernel; without
    it the vector variant runs.  The tuner's choice (either schedule) gives
    the same results again."""
    ws = members() if ragged else [w for w in members() if w.nx % 4 == 0]
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
    ens.set_schedule(schedule)
    for q, U in enumerate(states):
        ens.set_state(q, U)
    ens.step(dts, nsteps)
    info = ens.info()
    assert info["ctas"] > 0 and info["units"] > 0 and info["schedule"] == schedule
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


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_ensemble_member_matches_the_oracle(eb, oracle, precision):
    """Two members (a hill and a ragged random terrain) three steps in the
    ensemble against the FP64 oracle run on each member alone."""
    ws = [members()[0], members()[3]]
    geoms, states, dts, refs = [], [], [], []
    for q, w in enumerate(ws):
        r = refs_for(w.nz, w.Lz)
        refs.append(r)
        geoms.append(make_geometry(eb, w, w.heights(), precision, r))
        states.append(w.state("sheltered", seed=40 + q))
        dts.append(w.dt())
    ens = eb.Ensemble(geoms)
    for q in range(len(ws)):
        ens.set_state(q, to_device(states[q], precision, refs[q]))
    ens.step(dts, 3)
    for q, w in enumerate(ws):
        dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, w.heights())
        G = oracle.geometry(dom)
        want = oracle.step(dom, G, oracle.wsrd_setup(dom, G), states[q], dts[q], 3)
        got = to_host(ens.get_state(q), refs[q])
        act = active_masks(G, w.nz)
        for f in FIELDS:
            err = rel_linf(got[f], want[f], act[FGRID[f]])
            assert err <= TOL[precision], (precision, w.name, f, err)
    for g in geoms:
        eb.sync_status(g)
    ens.close()


def test_barrier_wait_expires_when_a_cta_never_arrives(eb):
    """CTA 0 of the persistent kernel skips the first grid barrier (the
    failure test's switch): every other CTA's bounded wait expires, the step
    returns and every member reports EB_ERR_TIMEOUT.  With the switch off
    again the next steps are exact (the barrier's counters are reset before
    every launch)."""
    ws = members()[:2]
    geoms = [make_geometry(eb, w, w.heights(), "mixed", refs_for(w.nz, w.Lz)) for w in ws]
    states = [to_device(w.state("sheltered", seed=3 + q), "mixed", refs_for(w.nz, w.Lz)) for q, w in enumerate(ws)]
    dts = [w.dt() for w in ws]
    want = [eb.step(g, U, dt, 2) for g, U, dt in zip(geoms, states, dts)]
    ens = eb.Ensemble(geoms)
    for q, U in enumerate(states):
        ens.set_state(q, U)
    ens.inject_barrier_fault(0)
    ens.step(dts, 1)
    for g in geoms:
        with pytest.raises(eb.EbError) as e:
            eb.sync_status(g)
        assert e.value.code == 5   # EB_ERR_TIMEOUT
    ens.inject_barrier_fault(-1)
    for q, U in enumerate(states):
        ens.set_state(q, U)
    ens.step(dts, 2)
    for q in range(len(ws)):
        got = ens.get_state(q)
        for f in FIELDS:
            assert torch.equal(got[f], want[q][f]), (ws[q].name, f)
    for g in geoms:
        eb.sync_status(g)
    with pytest.raises(eb.EbError):
        ens.inject_barrier_fault(ens.info()["ctas"])
    ens.close()
