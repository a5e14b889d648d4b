"""Shared helpers of the GPU tests: moving seeded states between numpy
(oracle) and torch (CUDA library), the relative L-inf error, and oracle runs
on column windows of large domains."""
import numpy as np

FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")
FGRID = {"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}

# Tolerances of the relative L-inf error (max |gpu - oracle| / max |oracle|
# over the compared CVs): the double path must agree to 1e-12, the mixed
# float path to 1e-5.
TOL = {"f64": 1e-12, "mixed": 1e-5}


# fields with a per-level profile, in the order of a refs tuple:
# (rho0, rho0 theta0) or (rho0, rho0 theta0, background rho*u, background rho*v)
REF_FIELDS = ("rho", "rhotheta", "rhou", "rhov")


def refs_for(nz, Lz):
    from paper_2604_11959_gb300 import inputs
    return inputs.cell_reference(nz, Lz)


def wind_refs(w, kind):
    """The stratified reference plus the background wind of state ``kind``."""
    return w.references(kind)


def _profile(refs, f):
    if refs is None or f not in REF_FIELDS:
        return None
    q = REF_FIELDS.index(f)
    return refs[q] if q < len(refs) else None


def to_device(U, precision, refs=None):
    """numpy full-value state -> torch CUDA state (perturbations about the
    per-level profiles in refs, where given)."""
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    out = {}
    for f in FIELDS:
        a = U[f]
        r = _profile(refs, f)
        if r is not None:
            a = a - np.asarray(r)[:, None, None]
        out[f] = torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    return out


def to_host(U, refs=None):
    out = {}
    for f in FIELDS:
        a = U[f].double().cpu().numpy()
        r = _profile(refs, f)
        if r is not None:
            a = a + np.asarray(r)[:, None, None]
        out[f] = a
    return out


def worst(got, want, mask):
    """Location and values of the largest difference (for messages)."""
    d = np.where(mask, np.abs(got - want), -1.0)
    loc = np.unravel_index(int(np.argmax(d)), d.shape)
    return {"at(k,j,i)": tuple(int(v) for v in loc), "got": float(got[loc]), "want": float(want[loc])}


def rel_linf(got, want, mask=None):
    d = np.abs(got - want)
    w = np.abs(want)
    if mask is not None:
        d, w = d[mask], w[mask]
    if d.size == 0:
        return 0.0
    den = w.max()
    return float(d.max() / den) if den > 0 else float(d.max())


def active_masks(G, nz):
    """Non-covered prognostic CVs per grid, from oracle geometry."""
    m = {}
    for g in range(4):
        a = G[g]["alpha"] > 0
        if g == 3:
            a = a.copy()
            a[0] = False
            a[nz] = False
        m[g] = a
    return m


def make_geometry(eb, w, h, precision, refs=None, vt=0.5):
    """A geometry handle; with a 4-entry refs tuple the background momenta
    are set too (eb_geom_set_wind_reference)."""
    import torch
    ht = torch.from_numpy(h).cuda()
    kw = {}
    if refs is not None:
        kw = dict(ref_rho=torch.from_numpy(refs[0]).cuda(), ref_rhotheta=torch.from_numpy(refs[1]).cuda())
        if len(refs) == 4:
            kw.update(ref_rhou=torch.from_numpy(np.ascontiguousarray(refs[2])).cuda(),
                      ref_rhov=torch.from_numpy(np.ascontiguousarray(refs[3])).cuda())
    return eb.Geometry(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, ht, precision=precision, v_target_frac=vt, **kw)


def window_oracle(oracle, w, h, U_full, x0, y0, W, dt, nsteps=1, stages=1):
    """Oracle run on a window of W x W columns at (x0, y0): geometry, tables
    and nsteps steps.  Returns (domain, geometry, tables, result)."""
    dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h, window=(x0, y0, W, W))
    G = oracle.geometry(dom)
    T = oracle.wsrd_setup(dom, G)
    Uw = {f: dom.window_of(U_full[f]) for f in FIELDS}
    R = oracle.step(dom, G, T, Uw, dt, nsteps, stages) if nsteps else Uw
    return dom, G, T, Uw, R


def window_cut(a, x0, y0, W, nx, ny):
    ii = (x0 + np.arange(W)) % nx
    jj = (y0 + np.arange(W)) % ny
    return a[..., jj[:, None], ii[None, :]]


def oracle_export(G, T, g, name):
    """The oracle's value of eb_geom_export field ``name`` of grid g
    (geometry G, redistribution tables T)."""
    if name == "alpha" or name == "aeb" or name == "flag":
        return G[g][name].astype(np.float64)
    if name.startswith("cent_") or name.startswith("nrm_") or name.startswith("ebc_") or name.startswith("beta_"):
        key, ax = name.split("_")
        return G[g][key]["xyz".index(ax)]
    if name.startswith("fcent_"):
        ax, t = name[6], int(name[7]) - 1
        return G[g]["fcent"][2 * "xyz".index(ax) + t]
    if name.startswith("xhat_"):
        return T[g]["xhat"]["xyz".index(name[5])]
    return T[g][name].astype(np.float64)
