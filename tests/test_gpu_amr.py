"""Two-level static refinement (Sec. 4.3) on the GPU against the oracle: the
coarse handle built from a fine one by merging its cells
(eb_geom_build_coarse) has the oracle's merged geometry and the redistribution
tables the oracle builds from it; steps on it match the oracle's steps on the
merged geometry; and eb_restrict matches the oracle's volume- and
area-weighted restriction.  A planar terrain's coarse handle equals the one
built directly from the coarse heights."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import (FGRID, FIELDS, TOL, active_masks, oracle_export, rel_linf, to_device, to_host, worst)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EXACT = ("flag", "code", "nnb")
CASES = {
    "grf": inputs.Workload("grf-48x40x24", 48, 40, 24, 1, terrain="grf", seed=5, hmax=0.2, tiny=3),
    "hill": inputs.Workload("hill-64x64x32", 64, 64, 32, 1, terrain="gaussian", hmax=0.15),
}


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11959_gb300 import build, eb as ebmod
    build.build()
    ebmod.load()
    return ebmod


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, oracle):
    w = CASES[request.param]
    h = w.heights()
    df = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h)
    Gf = oracle.geometry(df)
    dc = oracle.coarse_domain(df)
    Gc = oracle.coarsen(df, Gf, dc)
    Tc = oracle.wsrd_setup(dc, Gc)
    return request.param, w, h, df, Gf, dc, Gc, Tc


def _refs(nz, Lz):
    return inputs.cell_reference(nz, Lz)


def _handles(eb, w, h, precision):
    rf = _refs(w.nz, w.Lz)
    rc = _refs(w.nz // 2, w.Lz)
    fine = eb.Geometry(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, torch.from_numpy(h).cuda(), precision=precision,
                       ref_rho=torch.from_numpy(rf[0]).cuda(), ref_rhotheta=torch.from_numpy(rf[1]).cuda())
    coarse = fine.coarse(ref_rho=torch.from_numpy(rc[0]).cuda(), ref_rhotheta=torch.from_numpy(rc[1]).cuda())
    return fine, coarse, rf, rc


def _normal_weight(Gc, g, dc):
    """|sum_d (open area of the high d-face - of the low d-face) e_d| of every
    coarse CV of grid g over the largest face area: the length of the EB's
    area-weighted normal sum that the merged unit normal divides by (the high
    face of a CV is the next CV's low face; the lid above the top is open)."""
    return _weight_of(Gc[g]["beta"], (dc.dy * dc.dz, dc.dx * dc.dz, dc.dx * dc.dy))


def _weight_of(b, A):
    nv2 = np.zeros(b.shape[1:])
    for d in range(3):
        lo = b[d]
        if d < 2:
            hi = np.roll(lo, -1, axis=2 - d)
        else:
            hi = np.concatenate([lo[1:], np.ones((1,) + lo.shape[1:])], axis=0)
        nv2 += ((hi - lo) * A[d]) ** 2
    return np.sqrt(nv2) / max(A)


def test_coarse_geometry_and_tables_match(eb, case):
    """Every exported field of the coarse handle against the oracle's merged
    geometry and its tables: classes, codes and N exactly, moments and weights
    to 1e-12.  The unit EB normals are compared times the length of the
    area-weighted normal sum they are normalised from (a unit normal of a CV
    whose EB faces nearly cancel amplifies last-bit differences of the fine
    face fractions by its inverse)."""
    name, w, h, df, Gf, dc, Gc, Tc = case
    fine, coarse, _, _ = _handles(eb, w, h, "f64")
    assert (coarse.nx, coarse.ny, coarse.nz) == (w.nx // 2, w.ny // 2, w.nz // 2)
    for g in range(4):
        for f in eb.EXPORT_FIELDS:
            got = coarse.export(g, f).cpu().numpy()
            want = oracle_export(Gc, Tc, g, f)
            if f in EXACT:
                bad = np.argwhere(got != want)
                assert bad.size == 0, (name, g, f, bad[:5])
            else:
                d = np.abs(got - want)
                if f.startswith("nrm_"):
                    d = d * _normal_weight(Gc, g, dc)
                err = np.max(d)
                assert err <= 1e-12, (name, g, f, err, worst(got, want, np.ones(got.shape, bool)))
    info = coarse.info()
    assert info["cells"] == dc.NX * dc.NY * dc.nz
    assert sum(info["small_cvs"]) == sum(int((Tc[g]["code"] > 0).sum()) for g in range(4))
    fine.close()
    coarse.close()


@pytest.mark.parametrize("precision,stages", [("f64", 1), ("mixed", 1), ("f64", 3), ("mixed", 3)])
def test_steps_on_the_coarse_level_match(eb, case, oracle, precision, stages):
    """Steps of the coarse handle against the oracle's steps on the merged
    geometry (the sheltered state of the coarse grid)."""
    name, w, h, df, Gf, dc, Gc, Tc = case
    wc = inputs.Workload("coarse", w.nx // 2, w.ny // 2, w.nz // 2, 1, terrain=w.terrain, hmax=w.hmax)
    U = wc.state("sheltered", seed=4)
    dt = wc.dt()
    nsteps = 3 if stages == 1 else 2
    want = oracle.step(dc, Gc, Tc, U, dt, nsteps, stages)
    fine, coarse, _, rc = _handles(eb, w, h, precision)
    got = to_host(eb.step(coarse, to_device(U, precision, rc), dt, nsteps, stages), rc)
    eb.sync_status(coarse)
    act = active_masks(Gc, dc.nz)
    for f in FIELDS:
        err = rel_linf(got[f], want[f], act[FGRID[f]])
        assert err <= TOL[precision], (name, precision, stages, f, err)
    fine.close()
    coarse.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_restriction_matches(eb, case, oracle, precision):
    """A fine state (stored about the fine profiles) restricted onto the
    coarse level (stored about the coarse profiles) against the oracle's
    restriction of the full values; coarse CVs without fine fluid keep the
    value they had."""
    name, w, h, df, Gf, dc, Gc, Tc = case
    fine, coarse, rf, rc = _handles(eb, w, h, precision)
    Uf = w.state("sheltered", seed=6)
    wc = inputs.Workload("coarse", w.nx // 2, w.ny // 2, w.nz // 2, 1, terrain=w.terrain, hmax=w.hmax)
    U0 = wc.state("uniform", pert=1e-2, seed=7)
    want = oracle.restrict(df, Gf, Uf, dc, U0)
    Uc = to_device(U0, precision, rc)
    eb.restrict(fine, coarse, to_device(Uf, precision, rf), Uc)
    got = to_host(Uc, rc)
    tol = 1e-14 if precision == "f64" else 2e-7
    for f in FIELDS:
        err = rel_linf(got[f], want[f])
        assert err <= tol, (name, precision, f, err, worst(got[f], want[f], np.ones(got[f].shape, bool)))
    fine.close()
    coarse.close()


def test_planar_terrain_coarse_handle_equals_the_direct_one(eb):
    """On a planar terrain the merged coarse geometry is what the coarse
    heights give directly.  The EB normals are compared away from the
    periodic seam of the plane, where the faces of a CV come from both sides,
    and weighted as in test_coarse_geometry_and_tables_match."""
    NX, NY, nz = 32, 24, 16
    Lx, Ly, Lz = 1.0, 0.75, 0.5
    x = np.linspace(0, Lx, NX + 1)
    y = np.linspace(0, Ly, NY + 1)
    h = 0.123 + 0.21 * x[None, :] + 0.077 * y[:, None]
    fine = eb.Geometry(NX, NY, nz, Lx, Ly, Lz, torch.from_numpy(h).cuda(), precision="f64")
    coarse = fine.coarse()
    direct = eb.Geometry(NX // 2, NY // 2, nz // 2, Lx, Ly, Lz, torch.from_numpy(np.ascontiguousarray(h[::2, ::2])).cuda(),
                         precision="f64")
    dxc, dyc, dzc = 2 * Lx / NX, 2 * Ly / NY, 2 * Lz / nz
    for g in range(4):
        beta = np.stack([direct.export(g, f"beta_{a}").cpu().numpy() for a in "xyz"])
        wgt = _weight_of(beta, (dyc * dzc, dxc * dzc, dxc * dyc))[:, 1:-1, 1:-1]
        for f in ("alpha", "cent_x", "cent_y", "cent_z", "beta_x", "beta_y", "beta_z", "fcent_x1", "fcent_z2",
                  "aeb", "ebc_x", "ebc_z", "flag", "nrm_x", "nrm_z"):
            a = coarse.export(g, f).cpu().numpy()
            b = direct.export(g, f).cpu().numpy()
            d = np.abs(a - b)
            if f.startswith("nrm"):
                d = d[:, 1:-1, 1:-1] * wgt
            assert d.max() <= 1e-12, (g, f, float(d.max()))
    for q in (fine, coarse, direct):
        q.close()


def test_coarse_handle_argument_errors(eb):
    w = inputs.Workload("odd", 20, 18, 9, 1, terrain="gaussian", hmax=0.15)
    g = eb.Geometry(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, torch.from_numpy(w.heights()).cuda(), precision="f64")
    with pytest.raises(eb.EbError) as e:
        g.coarse()
    assert e.value.code == 1
    g.close()


@pytest.mark.parametrize("precision,stages", [("f64", 1), ("mixed", 1), ("f64", 3), ("mixed", 3)])
def test_two_level_steps_match(eb, oracle, precision, stages):
    """The coupled two-level step (paper_2604_11959_gb300/amr.py) against the
    same sequence in the oracle: a rough terrain with planted tiny cells,
    fine level 80x32x16, coarse level merged from it, one refined x-patch of
    16 fine columns; every step the patch's halo takes the coarse state, both
    levels advance with the fine time step, and the patch's owned columns are
    restricted onto the coarse level.  The whole coarse state and the patch's
    owned columns after three forward-Euler / two three-stage steps, both
    precisions, to 1e-12 / 1e-5."""
    from paper_2604_11959_gb300 import amr
    w = inputs.Workload("grf-80x32x16", 80, 32, 16, 1, terrain="grf", seed=9, hmax=0.2, tiny=2)
    wc = inputs.Workload("grf-40x16x8", 40, 16, 8, 1, Lx=w.Lx, Ly=w.Ly, Lz=w.Lz, terrain="grf", hmax=0.2)
    h = w.heights()
    H = amr.HALO_EULER if stages == 1 else amr.HALO_RK3
    x_lo, x_hi = 28, 44
    rf, rc = w.references("sheltered"), wc.references("sheltered")
    dt = w.dt()
    nsteps = 3 if stages == 1 else 2
    # oracle
    df = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h)
    dc = oracle.coarse_domain(df)
    Gc = oracle.coarsen(df, oracle.geometry(df), dc)
    Tc = oracle.wsrd_setup(dc, Gc)
    dw = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h, window=((x_lo - H) % w.nx, 0, x_hi - x_lo + 2 * H, w.ny))
    Gw = oracle.geometry(dw)
    Tw = oracle.wsrd_setup(dw, Gw)
    Uc = wc.state("sheltered", seed=3)
    grid = {"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}
    Uw = oracle.prolong(dc, Uc, dw, {f: np.zeros(dw.shape(grid[f])) for f in FIELDS}, (0, 0))
    # the library
    two = amr.TwoLevel(eb, w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h, x_lo, x_hi, H, precision, rf, rc)
    Cd = to_device(Uc, precision, rc)
    Fd = two.fill(Cd, two.patch.empty_state())
    for _ in range(nsteps):
        Uw = oracle.prolong(dc, Uc, dw, Uw, (x_lo, x_hi))
        Uc1 = oracle.step(dc, Gc, Tc, Uc, dt, 1, stages)
        Uw = oracle.step(dw, Gw, Tw, Uw, dt, 1, stages)
        Uc = oracle.restrict(dw, Gw, Uw, dc, Uc1, (x_lo, x_hi))
        Cd, Fd = two.step(Cd, Fd, dt, stages)
    eb.sync_status(two.coarse)
    eb.sync_status(two.patch)
    gc, gf = to_host(Cd, rc), to_host(Fd, rf)
    actc = active_masks(Gc, dc.nz)
    actw = active_masks(Gw, dw.nz)
    own = slice(H, H + x_hi - x_lo)
    for f in FIELDS:
        g = FGRID[f]
        err = rel_linf(gc[f], Uc[f], actc[g])
        assert err <= TOL[precision], ("coarse", precision, stages, f, err, worst(gc[f], Uc[f], actc[g]))
        a, b, m = gf[f][..., own], Uw[f][..., own], actw[g][..., own]
        err = rel_linf(a, b, m)
        assert err <= TOL[precision], ("patch", precision, stages, f, err, worst(a, b, m))
    two.close()
