"""Parity of the CUDA library (through the C ABI) with the FP64 CPU oracle.

Geometry flags, redistribution codes and neighbourhood counts must match bit
for bit; geometry moments and weights to 1e-12; state fields after N steps to
a relative L-inf error of 1e-12 (double path) or 1e-5 (mixed path)."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import (FGRID, FIELDS, TOL, active_masks, make_geometry, oracle_export, refs_for, rel_linf, to_device,
                          to_host, wind_refs, window_cut, window_oracle, worst)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EXACT = ("flag", "code", "nnb")


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11959_gb300 import build, eb as ebmod
    build.build()
    ebmod.load()
    return ebmod


def rough_workload():
    return inputs.Workload("grf-48x40x24", 48, 40, 24, 5, terrain="grf", seed=5, hmax=0.2, tiny=3)


CASES = {
    "woa": (inputs.WOA_32, None),
    "grf": (rough_workload(), None),
    "hill": (inputs.Workload("hill-64x64x32", 64, 64, 32, 10, terrain="gaussian", hmax=0.15), None),
    # odd nx and ny: rows not 16-byte aligned (element-wise copies in the bulk
    # kernel) and ragged tiles in both directions
    "odd": (inputs.Workload("grf-45x38x20", 45, 38, 20, 5, terrain="grf", seed=9, hmax=0.2, tiny=2), None),
    # the smallest grids: stencils wrap around the periodic boundaries several
    # times, one ragged tile holds the whole domain
    "tiny": (inputs.Workload("grf-6x5x4", 6, 5, 4, 3, terrain="grf", seed=11, hmax=0.2), None),
    # a steep, narrow hill (about ten levels per column): cut regions several
    # levels deep, so the redistribution reaches CVs the bulk kernel writes and
    # has to wait for it
    "steep": (inputs.Workload("steep-hill-32x32x32", 32, 32, 32, 3, terrain="gaussian", hmax=0.25, sigma=0.03), None),
}

# where every CV the redistribution touches is a near-EB CV, eb_step runs it
# beside the bulk kernel (set-up check); the steep hill is the case where it
# cannot
WSRD_BESIDE_BULK = {"woa": None, "grf": None, "hill": 1, "odd": None, "tiny": None, "steep": 0}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, oracle):
    w, _ = CASES[request.param]
    h = w.heights()
    dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h)
    G = oracle.geometry(dom)
    T = oracle.wsrd_setup(dom, G)
    return request.param, w, h, dom, G, T


def test_geometry_and_tables_match(eb, case):
    name, w, h, dom, G, T = case
    geom = make_geometry(eb, w, h, "f64")
    for g in range(4):
        for f in eb.EXPORT_FIELDS:
            got = geom.export(g, f).cpu().numpy()
            want = oracle_export(G, T, g, f)
            if f in EXACT:
                bad = np.argwhere(got != want)
                assert bad.size == 0, (name, g, f, bad[:5], got[tuple(bad[0])], want[tuple(bad[0])])
            else:
                err = np.max(np.abs(got - want))
                assert err <= 1e-12, (name, g, f, err, worst(got, want, np.ones(got.shape, bool)))
    info = geom.info()
    assert info["cells"] == w.nx * w.ny * w.nz
    for g in range(4):
        assert info["small_cvs"][g] == int((T[g]["code"] > 0).sum())


@pytest.mark.parametrize("precision,wind", [("f64", False), ("mixed", False), ("mixed", True)])
def test_flux_divergence_matches(eb, case, oracle, precision, wind):
    """dU of Eqs. update-cc / update-fc.  Compared volume weighted, alpha dU
    (the flux sum the update conserves): dU itself carries 1/alpha, which
    turns the last-bit differences of two independent geometry computations
    of a cell with alpha ~ 1e-13 into large relative differences.  With
    ``wind`` the state holds the momenta minus the background wind
    (eb_geom_set_wind_reference); dU is the same full derivative."""
    name, w, h, dom, G, T = case
    refs = wind_refs(w, "uniform") if wind else refs_for(w.nz, w.Lz)
    U = w.state("uniform", pert=1e-2, seed=11)
    want = oracle.flux_div(dom, G, U)
    geom = make_geometry(eb, w, h, precision, refs)
    got = to_host(eb.flux_div(geom, to_device(U, precision, refs)))
    act = active_masks(G, w.nz)
    for f in FIELDS:
        a = G[FGRID[f]]["alpha"]
        err = rel_linf(a * got[f], a * want[f], act[FGRID[f]])
        assert err <= TOL[precision], (name, precision, f, err, worst(a * got[f], a * want[f], act[FGRID[f]]))
        assert np.all(got[f][~act[FGRID[f]]] == 0.0)


def test_uniform_field_is_preserved_exactly(eb, case):
    """Redistribution of a constant returns it bit for bit (deviation form)."""
    name, w, h, dom, G, T = case
    geom = make_geometry(eb, w, h, "f64")
    for f in FIELDS:
        c = torch.full(geom.shape(f), 1.2345, dtype=torch.float64, device="cuda")
        assert torch.equal(eb.wsrd(geom, f, c), c), (name, f)
    geom32 = make_geometry(eb, w, h, "mixed")
    for f in ("rhou", "rhov", "rhow"):
        c = torch.full(geom32.shape(f), 0.75, dtype=torch.float32, device="cuda")
        assert torch.equal(eb.wsrd(geom32, f, c), c), (name, f)


@pytest.mark.parametrize("precision,wind", [("f64", False), ("mixed", False), ("f64", True), ("mixed", True)])
def test_redistribution_matches(eb, case, oracle, precision, wind):
    """Redistribution of every field; with ``wind`` the momenta are stored
    about a background profile and the redistribution adds the profile's
    level differences back (the oracle works on full values)."""
    name, w, h, dom, G, T = case
    refs = wind_refs(w, "sheltered") if wind else refs_for(w.nz, w.Lz)
    rng = np.random.default_rng(3)
    U = w.state("uniform", pert=0.05, seed=12)
    Uhat = {f: U[f] * (1.0 + 0.3 * rng.uniform(-1, 1, U[f].shape)) for f in FIELDS}
    geom = make_geometry(eb, w, h, precision, refs)
    dev = to_device(Uhat, precision, refs)
    act = active_masks(G, w.nz)
    for f in FIELDS:
        g = FGRID[f]
        want = oracle.wsrd(dom, G, T, g, Uhat[f])
        out = eb.wsrd(geom, f, dev[f])
        got = to_host({**{k: dev[k] for k in FIELDS}, f: out}, refs)[f]
        err = rel_linf(got, want, act[g])
        assert err <= TOL[precision], (name, precision, f, err, worst(got, want, act[g]))
        # CVs the redistribution does not touch are copied bit for bit
        untouched = act[g] & (T[g]["nnb"] == 1) & (T[g]["code"] == 0)
        assert np.array_equal(out.cpu().numpy()[untouched], dev[f].cpu().numpy()[untouched])


@pytest.mark.parametrize("precision,stages,kind,wind", [("f64", 1, "uniform", False), ("mixed", 1, "uniform", False),
                                                        ("mixed", 1, "uniform", True),
                                                        ("f64", 1, "sheltered", True), ("mixed", 1, "sheltered", True),
                                                        ("mixed", 1, "sheltered", False),
                                                        ("f64", 3, "sheltered", True), ("mixed", 3, "sheltered", True)])
def test_steps_match(eb, case, oracle, precision, stages, kind, wind):
    """Whole steps against the oracle.  ``wind``: the momenta are stored
    about the state's background wind (the configuration the benchmark
    runs), else as full values."""
    name, w, h, dom, G, T = case
    refs = wind_refs(w, kind) if wind else refs_for(w.nz, w.Lz)
    U = w.state(kind, pert=1e-2 if kind == "uniform" else 0.0, seed=21)
    # a uniform wind into the terrain (no pressure term) piles mass up on the
    # windward side and empties the lee cut cells within a few steps; already
    # at step 2 rounding the state to float moves the exact result by ~1e-5,
    # so uniform-wind runs stop after one step (two for double) and the
    # sheltered state runs the full step count
    if kind == "uniform":
        nsteps = 2 if precision == "f64" else 1
    else:
        nsteps = w.steps if stages == 1 else 3
    want = oracle.step(dom, G, T, U, w.dt(), nsteps, stages)
    geom = make_geometry(eb, w, h, precision, refs)
    got = to_host(eb.step(geom, to_device(U, precision, refs), w.dt(), nsteps, stages), refs)
    eb.sync_status(geom)
    act = active_masks(G, w.nz)
    for f in FIELDS:
        g = FGRID[f]
        err = rel_linf(got[f], want[f], act[g])
        assert err <= TOL[precision], (name, precision, stages, kind, f, err, worst(got[f], want[f], act[g]))
        # covered CVs and the w wall levels pass through unchanged
        static = ~act[g]
        ref_in = to_host(to_device({k: U[k] for k in FIELDS}, precision, refs), refs)[f]
        assert np.array_equal(got[f][static], ref_in[static]), (name, f)


def test_redistribution_schedule(eb, case):
    """The set-up check that lets the redistribution run beside the bulk kernel
    gives the expected answer on the cases where it is known; the steps of
    every case match the oracle either way (test_steps_match)."""
    name, w, h, dom, G, T = case
    geom = make_geometry(eb, w, h, "f64", refs_for(w.nz, w.Lz))
    flag = geom.info()["wsrd_beside_bulk"]
    assert flag in (0, 1)
    if WSRD_BESIDE_BULK[name] is not None:
        assert flag == WSRD_BESIDE_BULK[name], (name, flag)
    geom.close()


def test_deterministic(eb):
    w = rough_workload()
    h = w.heights()
    U = w.state("uniform", pert=1e-2, seed=4)
    geom = make_geometry(eb, w, h, "mixed", refs_for(w.nz, w.Lz))
    a = eb.step(geom, to_device(U, "mixed", refs_for(w.nz, w.Lz)), w.dt(), 4)
    b = eb.step(geom, to_device(U, "mixed", refs_for(w.nz, w.Lz)), w.dt(), 4)
    for f in FIELDS:
        assert torch.equal(a[f], b[f]), f


# ---------------------------------------------------------------------------
# full-size workloads: the launch configuration the benchmark times, checked
# on column windows that the oracle computes one by one
# ---------------------------------------------------------------------------
FULL = {"hill256": inputs.HILL_256, "grf512": inputs.GRF_512}


@pytest.mark.parametrize("which", sorted(FULL))
@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_full_size_windows(eb, oracle, which, precision):
    w = FULL[which]
    h = w.heights()
    refs = wind_refs(w, "uniform")
    U = w.state("uniform", pert=1e-2, seed=31)
    geom = make_geometry(eb, w, h, precision, refs)
    got = to_host(eb.step(geom, to_device(U, precision, refs), w.dt(), 1, 1), refs)
    eb.sync_status(geom)
    exp_flag = {g: geom.export(g, "flag").cpu().numpy() for g in range(4)}
    exp_code = {g: geom.export(g, "code").cpu().numpy() for g in range(4)}
    W, M = 34, 10
    rng = np.random.default_rng(5)
    # windows: the highest terrain column, a planted tiny cell (if any) and two random spots
    hj, hi = np.unravel_index(np.argmax(h[:-1, :-1]), (w.ny, w.nx))
    spots = [(hi, hj)] + [(int(rng.integers(0, w.nx)), int(rng.integers(0, w.ny))) for _ in range(2)]
    if w.tiny:
        _, planted = inputs.plant_tiny_cells(inputs.grf_terrain(w.nx, w.ny, w.seed, w.hmax), w.nx, w.ny, w.nz, w.Lz,
                                             w.tiny, w.seed + 1)
        spots.append(planted[0][:2])
    for (ci, cj) in spots:
        x0, y0 = (ci - W // 2) % w.nx, (cj - W // 2) % w.ny
        dom, G, T, Uw, R = window_oracle(oracle, w, h, U, x0, y0, W, w.dt(), 1, 1)
        inner = (slice(None), slice(M, W - M), slice(M, W - M))
        for g in range(4):
            wf = window_cut(exp_flag[g], x0, y0, W, w.nx, w.ny)
            bad = np.argwhere(wf[inner] != G[g]["flag"][inner])
            assert bad.size == 0, (which, g, (x0, y0), bad[:3], wf[inner][tuple(bad[0])],
                                   G[g]["flag"][inner][tuple(bad[0])])
            wc = window_cut(exp_code[g], x0, y0, W, w.nx, w.ny)
            assert np.array_equal(wc[inner], T[g]["code"][inner].astype(np.float64)), (which, g)
        act = active_masks(G, w.nz)
        for f in FIELDS:
            g = FGRID[f]
            gw = window_cut(got[f], x0, y0, W, w.nx, w.ny)
            m = act[g].copy()
            m[:, :M, :] = False
            m[:, W - M:, :] = False
            m[:, :, :M] = False
            m[:, :, W - M:] = False
            err = rel_linf(gw, R[f], m)
            assert err <= TOL[precision], (which, precision, (ci, cj), f, err)


# ---------------------------------------------------------------------------
# error handling
# ---------------------------------------------------------------------------
def test_invalid_arguments(eb):
    w = inputs.WOA_32
    h = torch.from_numpy(w.heights()).cuda()
    with pytest.raises(eb.EbError) as e:
        eb.Geometry(2, w.ny, w.nz, 1.0, 1.0, 0.5, torch.zeros((w.ny + 1, 3), dtype=torch.float64, device="cuda"))
    assert e.value.code == 1
    geom = eb.Geometry(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h)
    U = to_device(w.state("uniform"), "f64")
    with pytest.raises(eb.EbError) as e:
        eb.step(geom, U, -1.0, 1)
    assert e.value.code == 1
    with pytest.raises(eb.EbError) as e:
        eb.step(geom, U, w.dt(), 1, stages=2)
    assert e.value.code == 1
    with pytest.raises(eb.EbError) as e:
        eb.step(geom, U, w.dt(), 1, out=U)
    assert e.value.code == 1


def test_non_finite_state_is_reported(eb):
    w = inputs.WOA_32
    geom = make_geometry(eb, w, w.heights(), "mixed", refs_for(w.nz, w.Lz))
    U = to_device(w.state("uniform"), "mixed", refs_for(w.nz, w.Lz))
    U["rhou"][12, 5, 7] = float("nan")
    eb.step(geom, U, w.dt(), 1)
    with pytest.raises(eb.EbError) as e:
        eb.sync_status(geom)
    assert e.value.code == 4
    eb.sync_status(geom)   # cleared


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_tuning_changes_no_result(eb, precision):
    """eb_geom_tune only re-splits the bulk kernel's columns into slabs: every
    cell's arithmetic is the same, so steps after tuning equal the steps before
    it bit for bit, and the tuner leaves its input state untouched."""
    w = rough_workload()
    refs = refs_for(w.nz, w.Lz)
    U = w.state("uniform", pert=1e-2, seed=6)
    geom = make_geometry(eb, w, w.heights(), precision, refs)
    A = to_device(U, precision, refs)
    before = eb.step(geom, A, w.dt(), 3)
    keep = {f: A[f].clone() for f in A}
    best = eb.tune(geom, A, w.dt(), reps=1)
    assert best in (0, 12, 16, 24, 32, 48, 64, w.nz)
    info = geom.info()
    assert info["slab_levels"] == best and info["bulk_high_priority"] in (0, 1)
    for f in A:
        assert torch.equal(A[f], keep[f]), f
    after = eb.step(geom, A, w.dt(), 3)
    for f in FIELDS:
        assert torch.equal(before[f], after[f]), (precision, f)
    eb.sync_status(geom)
    geom.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_every_slab_height_gives_the_same_steps(eb, precision):
    """The bulk kernel's slab heights (eb_geom_set_slab_levels: automatic,
    a few levels, whole columns) and tile heights (eb_geom_set_tile_rows: 16,
    or 14 on the mixed path) change which CTA marches which columns and
    levels, never a cell's arithmetic: the steps agree bit for bit, and other
    values are rejected."""
    w = rough_workload()
    refs = refs_for(w.nz, w.Lz)
    U = w.state("uniform", pert=1e-2, seed=6)
    geom = make_geometry(eb, w, w.heights(), precision, refs)
    A = to_device(U, precision, refs)
    eb.set_slab_levels(geom, 0)
    want = eb.step(geom, A, w.dt(), 3)
    for rows in ((16, 14) if precision == "mixed" else (16,)):
        eb.set_tile_rows(geom, rows)
        assert geom.info()["tile_rows"] == rows
        for split in (0, 1, 5, w.nz + 7):
            eb.set_slab_levels(geom, split)
            assert geom.info()["slab_levels"] == split
            got = eb.step(geom, A, w.dt(), 3)
            for f in FIELDS:
                assert torch.equal(got[f], want[f]), (precision, rows, split, f)
    with pytest.raises(eb.EbError):
        eb.set_slab_levels(geom, -1)
    with pytest.raises(eb.EbError):
        eb.set_tile_rows(geom, 15)
    if precision == "f64":
        with pytest.raises(eb.EbError):
            eb.set_tile_rows(geom, 14)
    eb.sync_status(geom)
    geom.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_bulk_priority_changes_no_result(eb, precision):
    """The bulk kernel on the high-priority stream or on the caller's stream
    (eb_geom_set_bulk_priority) only changes the schedule: the steps agree
    bit for bit, the choice shows in eb_geom_info, and other values are
    rejected."""
    w = rough_workload()
    refs = refs_for(w.nz, w.Lz)
    U = w.state("uniform", pert=1e-2, seed=7)
    geom = make_geometry(eb, w, w.heights(), precision, refs)
    A = to_device(U, precision, refs)
    eb.set_bulk_priority(geom, False)
    assert geom.info()["bulk_high_priority"] == 0
    low = eb.step(geom, A, w.dt(), 3)
    eb.set_bulk_priority(geom, True)
    assert geom.info()["bulk_high_priority"] == 1
    high = eb.step(geom, A, w.dt(), 3)
    for f in FIELDS:
        assert torch.equal(low[f], high[f]), (precision, f)
    assert eb.load().eb_geom_set_bulk_priority(geom.handle, 2) == 1   # EB_ERR_INVALID_ARG
    eb.sync_status(geom)
    geom.close()


def test_packed_state_gives_the_same_step(eb):
    """A state held in one allocation (Geometry.packed_state: per-field views,
    each on a 256-byte boundary) steps exactly like separate tensors."""
    w = rough_workload()
    refs = refs_for(w.nz, w.Lz)
    geom = make_geometry(eb, w, w.heights(), "mixed", refs)
    A = to_device(w.state("uniform", pert=1e-2, seed=8), "mixed", refs)
    flat, views = geom.packed_state()
    for f in FIELDS:
        views[f].copy_(A[f])
        assert views[f].data_ptr() % 256 == 0
    oflat, oviews = geom.packed_state()
    want = eb.step(geom, A, w.dt(), 2)
    eb.step(geom, views, w.dt(), 2, out=oviews)
    for f in FIELDS:
        assert torch.equal(want[f], oviews[f]), f
    geom.close()


def test_wind_reference_zero_is_full_values(eb):
    """A zero background profile (set explicitly) steps bit for bit like no
    profile; a nonzero profile with the state shifted by it gives the same
    full result to float rounding after one step (the two float paths round
    differently, and on this uniform wind into the terrain their difference
    grows past 1e-5 from the second step on, as each one's error against the
    oracle does); the anelastic calls refuse a handle with a profile (they
    need full momenta)."""
    w = rough_workload()
    refs = refs_for(w.nz, w.Lz)
    U = w.state("uniform", pert=1e-2, seed=9)
    g0 = make_geometry(eb, w, w.heights(), "mixed", refs)
    want = eb.step(g0, to_device(U, "mixed", refs), w.dt(), 2)
    zero = torch.zeros(w.nz, dtype=torch.float64, device="cuda")
    g0.set_wind_reference(zero, zero)
    got = eb.step(g0, to_device(U, "mixed", refs), w.dt(), 2)
    for f in FIELDS:
        assert torch.equal(want[f], got[f]), f
    wr = wind_refs(w, "uniform")
    g1 = make_geometry(eb, w, w.heights(), "mixed", wr)
    full = to_host(eb.step(g1, to_device(U, "mixed", wr), w.dt(), 1), wr)
    base = to_host(eb.step(g0, to_device(U, "mixed", refs), w.dt(), 1), refs)
    for f in FIELDS:
        assert rel_linf(full[f], base[f]) <= TOL["mixed"], f
    with pytest.raises(eb.EbError) as e:
        eb.project(g1, to_device(U, "mixed", wr), w.dt())
    assert e.value.code == 6   # EB_ERR_STATE
    g0.close()
    g1.close()
