"""Pins of the oracle's two-level refinement operators (Sec. 4.3; section 6
of oracle/eb_oracle.c): the coarse level's geometry merged from the fine
level's cells, and the restriction of a fine state.  Each pin fails on a
named mutation, given in its docstring."""
import numpy as np

from paper_2604_11959_gb300 import inputs

FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")
KEYS = ("alpha", "cent", "beta", "fcent", "aeb", "nrm", "ebc", "ebv", "flag")


def _planar(oracle):
    NX, NY, nz = 16, 12, 12
    Lx, Ly, Lz = 1.0, 0.75, 0.5
    x = np.linspace(0, Lx, NX + 1)
    y = np.linspace(0, Ly, NY + 1)
    h = 0.123 + 0.21 * x[None, :] + 0.077 * y[:, None]
    return oracle.Domain(NX, NY, nz, Lx, Ly, Lz, h)


def _rough(oracle):
    w = inputs.Workload("grf-32x24x16", 32, 24, 16, 1, terrain="grf", seed=7, hmax=0.22, tiny=3)
    return oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, w.heights())


def test_planar_terrain_merges_to_the_direct_coarse_geometry(oracle):
    """A plane is represented exactly on both levels, so merging the fine
    cells must give what the coarse geometry computes directly from the
    plane: every moment of the four grids to 1e-12, the classes exactly.  The
    EB normals are compared away from the periodic seam of the (non-periodic)
    plane, where a CV's faces come from both sides of the seam.  Fails if the
    fine offsets are not halved into coarse units, if the u, v or w grid
    merges cells 2I, 2I+1 instead of 2I-1, 2I, if the EB area is not quartered,
    or if the normal takes the low-minus-high face areas."""
    df = _planar(oracle)
    Gf = oracle.geometry(df)
    dc = oracle.coarse_domain(df)
    merged = oracle.coarsen(df, Gf, dc)
    direct = oracle.geometry(dc)
    for g in range(4):
        assert (direct[g]["flag"] == 2).sum() > 50
        for k in KEYS:
            a, b = merged[g][k].astype(float), direct[g][k].astype(float)
            if k == "nrm":
                a, b = a[..., 1:-1, 1:-1], b[..., 1:-1, 1:-1]
            assert np.abs(a - b).max() <= 1e-12, (g, k, float(np.abs(a - b).max()))


def _blocks(a, g, nz_f):
    """Fine c-grid array (nz_f, NY, NX) -> (Kc, Jc, Ic, 2, 2, 2) blocks of the
    coarse CVs of grid g (cells outside the domain in z are zero)."""
    sx, sy, sz = g == 1, g == 2, g == 3
    pad = np.zeros((nz_f + 2,) + a.shape[1:])
    pad[1:-1] = a
    a = np.roll(np.roll(pad, int(sx), axis=2), int(sy), axis=1)   # cell 2I - s sits at index 2I
    a = a[1 - int(sz):] if sz else a[1:]
    K = (nz_f // 2) + (1 if g == 3 else 0)
    a = a[:2 * K]
    return a.reshape(K, 2, a.shape[1] // 2, 2, a.shape[2] // 2, 2).transpose(0, 2, 4, 1, 3, 5)


def test_volumes_and_areas_are_sums_of_fine_ones(oracle):
    """On a rough terrain with planted tiny cells: every coarse volume
    fraction is the mean of its 8 fine cells, every coarse low-face fraction
    the mean of the 4 fine faces on it, every EB area a quarter of the fine
    sum, and the class is covered / regular exactly when all fine cells are.
    Fails on a wrong block (cells 2I, 2I+1 for a face grid), on a missing
    normalisation, or on the class of a partly covered block."""
    df = _rough(oracle)
    Gf = oracle.geometry(df)
    dc = oracle.coarse_domain(df)
    Gc = oracle.coarsen(df, Gf, dc)
    F = Gf[0]
    for g in range(4):
        al = _blocks(F["alpha"], g, df.nz)
        assert np.abs(Gc[g]["alpha"] - al.sum(axis=(3, 4, 5)) / 8).max() <= 1e-15
        ae = _blocks(F["aeb"], g, df.nz)
        assert np.abs(Gc[g]["aeb"] - ae.sum(axis=(3, 4, 5)) / 4).max() <= 1e-14
        for d in range(3):
            be = _blocks(F["beta"][d], g, df.nz)
            low = np.take(be, 0, axis=3 + (2 - d))   # the fine cells on the coarse low d-face
            assert np.abs(Gc[g]["beta"][d] - low.sum(axis=(3, 4)) / 4).max() <= 1e-15, (g, d)
        fl = _blocks(F["flag"].astype(float) + 10.0, g, df.nz)     # 0 marks a cell outside the domain
        inside = fl > 0
        cov = ((fl == 10.0) | ~inside).all(axis=(3, 4, 5))
        reg = ((fl == 11.0) | ~inside).all(axis=(3, 4, 5))
        want = np.where(cov, 0, np.where(reg, 1, 2))
        assert np.array_equal(Gc[g]["flag"], want), g


def test_restriction_keeps_totals_and_uniform_states(oracle):
    """Restricting a random fine state: every coarse cell holds the volume-
    weighted total of its fine cells (sum alpha U over the 8 = 8 alpha_c U_c)
    and every coarse face the area-weighted flux integral of its 4 fine faces
    (sum beta U = 4 beta_c U_c); a uniform fine state restricts to the same
    uniform state; coarse CVs with no fine fluid keep their values.  Fails on
    plain (unweighted) means, on the face grids taking the fine faces 2I + 1,
    or on weights from the wrong face direction."""
    df = _rough(oracle)
    Gf = oracle.geometry(df)
    dc = oracle.coarse_domain(df)
    Gc = oracle.coarsen(df, Gf, dc)
    rng = np.random.default_rng(3)
    grid = {"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}
    Uf = {f: 1.0 + rng.random(df.shape(grid[f])) for f in FIELDS}
    keep = {f: np.full(dc.shape(3 if f == "rhow" else 0), -7.0) for f in FIELDS}
    R = oracle.restrict(df, Gf, Uf, dc, keep)
    F = Gf[0]
    for f in ("rho", "rhotheta"):
        tot = _blocks(F["alpha"] * Uf[f], 0, df.nz).sum(axis=(3, 4, 5))
        fluid = Gc[0]["alpha"] > 0
        assert np.abs(8 * Gc[0]["alpha"] * R[f] - tot)[fluid].max() <= 1e-13 * np.abs(tot).max()
        assert (R[f][~fluid] == -7.0).all()
    for f, d in (("rhou", 0), ("rhov", 1)):
        # the fine faces at fine index 2I: the low d-faces of the fine cells 2I
        be = F["beta"][d]
        s = (be * Uf[f]).reshape(df.nz // 2, 2, df.NY // 2, 2, df.NX // 2, 2)
        b4 = be.reshape(df.nz // 2, 2, df.NY // 2, 2, df.NX // 2, 2)
        if d == 0:
            s, b4 = s[:, :, :, :, :, 0], b4[:, :, :, :, :, 0]
        else:
            s, b4 = s[:, :, :, 0, :, :], b4[:, :, :, 0, :, :]
        tot = s.sum(axis=(1, 3)) if d == 0 else s.sum(axis=(1, 4))
        wsum = b4.sum(axis=(1, 3)) if d == 0 else b4.sum(axis=(1, 4))
        open_ = wsum > 0
        assert np.abs(wsum * R[f] - tot)[open_].max() <= 1e-13 * np.abs(tot).max(), f
        assert np.allclose(wsum / 4, Gc[0]["beta"][d]), f   # the coarse cell face itself
    U1 = {f: np.full_like(Uf[f], 2.5) for f in FIELDS}
    R1 = oracle.restrict(df, Gf, U1, dc, keep)
    for f in FIELDS:
        m = R1[f] != -7.0
        assert m.any() and np.abs(R1[f][m] - 2.5).max() <= 1e-15, f


def test_prolongation_then_restriction_is_the_identity(oracle):
    """Prolonging a coarse state onto a fine window (every column not owned)
    and restricting it back gives the coarse state on every coarse CV with fine
    fluid: injected cell values and face values on coarse faces are kept by
    the weighted means.  A face field linear along its axis is prolonged
    exactly (the odd fine faces take the mean of their two coarse faces), and
    owned columns are left alone.  Fails if the odd faces take one neighbour,
    if cells take a neighbouring coarse cell, or if owned columns are
    overwritten."""
    df = _rough(oracle)
    dc = oracle.coarse_domain(df)
    Gf = oracle.geometry(df)
    rng = np.random.default_rng(5)
    grid = {"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}
    Uc = {f: 1.0 + rng.random(dc.shape(grid[f])) for f in FIELDS}
    Uc["rhou"] = np.broadcast_to(0.3 * np.arange(dc.NX)[None, None, :], dc.shape(1)).copy() + 1.0
    win = oracle.Domain(df.NX, df.NY, df.nz, df.Lx, df.Ly, df.Lz, df.h, window=(8, 0, 20, df.NY))
    U0 = {f: np.full(win.shape(grid[f]), -3.0) for f in FIELDS}
    owned = (12, 24)                               # global fine columns 12 .. 23 of the window 8 .. 27
    P = oracle.prolong(dc, Uc, win, U0, owned)
    for f in FIELDS:
        assert (P[f][..., 4:16] == -3.0).all(), f  # owned columns untouched
        assert (P[f][..., :4] != -3.0).all() and (P[f][..., 16:] != -3.0).all(), f
    # rho*u linear in the coarse face index: fine face 2I + 1 sits halfway
    xi = 8 + np.arange(20)
    want = 1.0 + 0.3 * (xi / 2.0)
    halo = np.r_[0:4, 16:20]
    assert np.abs(P["rhou"][..., halo] - want[halo]).max() <= 1e-14
    full = {f: oracle.prolong(dc, Uc, df, {k: np.zeros(df.shape(grid[k])) for k in FIELDS}, (0, 0))[f]
            for f in FIELDS}
    back = oracle.restrict(df, Gf, full, dc, {f: np.full(dc.shape(grid[f]), -9.0) for f in FIELDS})
    for f in FIELDS:
        m = back[f] != -9.0
        assert m.sum() > 0.5 * m.size, f
        assert np.abs(back[f][m] - Uc[f][m]).max() <= 1e-14 * np.abs(Uc[f]).max(), f
