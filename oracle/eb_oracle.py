"""ctypes front end of the FP64 CPU oracle in ``eb_oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The oracle shares no
code with the CUDA library and never imports it.

Arrays are numpy, shaped ``(nz_g, WY, WX)`` (x fastest) for a grid with
``nz_g`` levels (``nz`` for the c, u and v grids, ``nz + 1`` for w).  Vector
fields carry a leading axis of 3 (or 6 for face centroids).

The step follows Algorithm 1 of the paper: ``stages=1`` is the forward-Euler
update of Eq. FV-discrete, ``stages=3`` the three-stage Runge-Kutta of Sec.
5.2 (U1 = U + dt/3 L(U), U2 = U + dt/2 L(U1), U' = U + dt L(U2)) with
redistribution after every stage; L is the flux divergence, plus the sources
of the compressible system (Sec. 2.1: the perturbation pressure gradient from
the equation of state and the buoyancy) when a ``Sources`` is given.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libeb_oracle.so")

GRIDS = ("c", "u", "v", "w")
FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")
FIELD_GRID = {"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}
COVERED, REGULAR, CUT = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP if present)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _SO + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


class _Domain(ctypes.Structure):
    _fields_ = [("NX", ctypes.c_int), ("NY", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_int), ("y0", ctypes.c_int), ("WX", ctypes.c_int), ("WY", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("h", ctypes.c_void_p)]


class _Geom(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("alpha", "cent", "beta", "fcent", "aeb", "nrm", "ebc", "ebv", "flag")]


class _Wsrd(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("code", "nnb", "kappa", "omega", "vhat", "xhat")]


class _State(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p * 5)]


class _Sources(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_void_p), ("rt0", ctypes.c_void_p), ("grav", ctypes.c_double),
                ("pressure", ctypes.c_int), ("buoyancy", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.orc_geometry.argtypes = [P(_Domain), ctypes.c_int, P(_Geom)]
            lib.orc_wsrd_setup.argtypes = [P(_Domain), ctypes.c_int, P(_Geom), ctypes.c_double, P(_Wsrd)]
            lib.orc_flux_div.argtypes = [P(_Domain), P(_Geom), P(_State), P(_State)]
            lib.orc_wsrd_apply.argtypes = [P(_Domain), ctypes.c_int, P(_Geom), P(_Wsrd), ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_stage.argtypes = [P(_Domain), P(_Geom), P(_Wsrd), P(_State), P(_State), ctypes.c_double,
                                      P(_State), P(_State), P(_Sources)]
            lib.orc_sources.argtypes = [P(_Domain), P(_Geom), P(_State), P(_Sources), P(_State)]
            lib.orc_coarsen.argtypes = [P(_Domain), P(_Geom), P(_Domain), ctypes.c_int, P(_Geom)]
            lib.orc_restrict.argtypes = [P(_Domain), P(_Geom), P(_State), P(_Domain), P(_State), ctypes.c_int,
                                         ctypes.c_int]
            lib.orc_prolong.argtypes = [P(_Domain), P(_State), P(_Domain), P(_State), ctypes.c_int, ctypes.c_int]
            lib.orc_eos_pressure.argtypes = [ctypes.c_double]
            lib.orc_eos_pressure.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class Domain:
    """A periodic NX x NY x nz grid on [0,Lx]x[0,Ly]x[0,Lz] with nodal terrain
    ``h`` of shape (NY+1, NX+1); arrays cover the window of columns
    [x0, x0+WX) x [y0, y0+WY) (default: the whole domain)."""

    def __init__(self, NX, NY, nz, Lx, Ly, Lz, h, window=None):
        self.NX, self.NY, self.nz = int(NX), int(NY), int(nz)
        self.Lx, self.Ly, self.Lz = float(Lx), float(Ly), float(Lz)
        self.dx, self.dy, self.dz = self.Lx / self.NX, self.Ly / self.NY, self.Lz / self.nz
        self.h = np.ascontiguousarray(h, dtype=np.float64)
        assert self.h.shape == (self.NY + 1, self.NX + 1)
        if window is None:
            window = (0, 0, self.NX, self.NY)
        self.x0, self.y0, self.WX, self.WY = (int(v) for v in window)
        assert 0 < self.WX <= self.NX and 0 < self.WY <= self.NY
        self._c = _Domain(self.NX, self.NY, self.nz, self.x0, self.y0, self.WX, self.WY,
                          self.dx, self.dy, self.dz, _ptr(self.h))

    def nzg(self, g: int) -> int:
        return self.nz + (1 if g == 3 else 0)

    def shape(self, g: int):
        return (self.nzg(g), self.WY, self.WX)

    def window_of(self, arr: np.ndarray) -> np.ndarray:
        """Cut this domain's window out of a global (nz_g, NY, NX) array, with
        periodic wrap."""
        ii = (self.x0 + np.arange(self.WX)) % self.NX
        jj = (self.y0 + np.arange(self.WY)) % self.NY
        return np.ascontiguousarray(arr[..., jj[:, None], ii[None, :]])


def geometry(dom: Domain) -> dict:
    """Geometry of the four grids (Sec. 3.2) as dicts of arrays."""
    lib = _load()
    out = {}
    for g in range(4):
        s = dom.shape(g)
        G = dict(alpha=np.zeros(s), cent=np.zeros((3,) + s), beta=np.zeros((3,) + s),
                 fcent=np.zeros((6,) + s), aeb=np.zeros(s), nrm=np.zeros((3,) + s),
                 ebc=np.zeros((3,) + s), ebv=np.zeros((3,) + s), flag=np.zeros(s, np.uint8))
        cg = _Geom(*(_ptr(G[k]) for k in ("alpha", "cent", "beta", "fcent", "aeb", "nrm", "ebc", "ebv", "flag")))
        lib.orc_geometry(ctypes.byref(dom._c), g, ctypes.byref(cg))
        out[g] = G
    return out


def _cgeom(geom):
    arr = (_Geom * 4)()
    for g in range(4):
        G = geom[g]
        arr[g] = _Geom(*(_ptr(G[k]) for k in ("alpha", "cent", "beta", "fcent", "aeb", "nrm", "ebc", "ebv", "flag")))
    return arr


def wsrd_setup(dom: Domain, geom: dict, vt: float = 0.5) -> dict:
    """Merging neighbourhoods and weights of every grid (Sec. 5.1)."""
    lib = _load()
    out = {}
    cg = _cgeom(geom)
    for g in range(4):
        s = dom.shape(g)
        T = dict(code=np.zeros(s, np.uint8), nnb=np.zeros(s, np.int32), kappa=np.zeros(s), omega=np.zeros(s),
                 vhat=np.zeros(s), xhat=np.zeros((3,) + s))
        cw = _Wsrd(*(_ptr(T[k]) for k in ("code", "nnb", "kappa", "omega", "vhat", "xhat")))
        lib.orc_wsrd_setup(ctypes.byref(dom._c), g, ctypes.byref(cg[g]), float(vt), ctypes.byref(cw))
        out[g] = T
    return out


def _cstate(U):
    st = _State()
    for f, name in enumerate(FIELDS):
        st.f[f] = _ptr(U[name])
    return st


def _check_state(dom, U):
    for name in FIELDS:
        a = U[name]
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], name
        assert a.shape == dom.shape(FIELD_GRID[name]), (name, a.shape)


def empty_state(dom: Domain) -> dict:
    return {n: np.zeros(dom.shape(FIELD_GRID[n])) for n in FIELDS}


def flux_div(dom: Domain, geom: dict, U: dict) -> dict:
    """dU of Eqs. update-cc / update-fc for every prognostic non-covered CV."""
    _check_state(dom, U)
    lib = _load()
    dU = empty_state(dom)
    lib.orc_flux_div(ctypes.byref(dom._c), _cgeom(geom), ctypes.byref(_cstate(U)), ctypes.byref(_cstate(dU)))
    return dU


def wsrd(dom: Domain, geom: dict, tabs: dict, g: int, Uhat: np.ndarray, diag: bool = False):
    """Redistribution of one field on grid g (Eqs. qhat_omega .. final_update_omega).
    With ``diag`` also the limited slopes sigma (3, ...), the limiter factors
    phi and the neighbourhood averages Qhat of every CV (Uhat where the CV is
    not small)."""
    lib = _load()
    Uhat = np.ascontiguousarray(Uhat, dtype=np.float64)
    assert Uhat.shape == dom.shape(g)
    out = np.empty_like(Uhat)
    cg = _cgeom(geom)
    T = tabs[g]
    cw = _Wsrd(*(_ptr(T[k]) for k in ("code", "nnb", "kappa", "omega", "vhat", "xhat")))
    sig = np.zeros((3,) + Uhat.shape) if diag else None
    phi = np.zeros(Uhat.shape) if diag else None
    qh = np.zeros(Uhat.shape) if diag else None
    lib.orc_wsrd_apply(ctypes.byref(dom._c), g, ctypes.byref(cg[g]), ctypes.byref(cw), _ptr(Uhat), _ptr(out),
                       _ptr(sig) if diag else None, _ptr(phi) if diag else None, _ptr(qh) if diag else None)
    if diag:
        return out, sig, phi, qh
    return out


class Sources:
    """The sources of the compressible system (Sec. 2.1, Eq. mom-comp) for a
    reference state given per level: rho0 and rho0*theta0 (nz values each);
    ``pressure``: -grad p' with p from the equation of state, ``buoyancy``:
    -rho' g on rho*w."""

    def __init__(self, rho0, rt0, pressure=True, buoyancy=True, grav=9.81):
        self.rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
        self.rt0 = np.ascontiguousarray(rt0, dtype=np.float64)
        self.pressure, self.buoyancy, self.grav = bool(pressure), bool(buoyancy), float(grav)

    def _c(self):
        return _Sources(_ptr(self.rho0), _ptr(self.rt0), self.grav, int(self.pressure), int(self.buoyancy))


def eos_pressure(rt: float) -> float:
    """p of the equation of state for rho*theta = rt (Sec. 2.1)."""
    return float(_load().orc_eos_pressure(float(rt)))


def sources(dom: Domain, geom: dict, U: dict, S: Sources) -> dict:
    """The sources of state U alone, as a dU (zero on the c grid)."""
    _check_state(dom, U)
    assert S.rho0.shape == (dom.nz,) and S.rt0.shape == (dom.nz,)
    dU = empty_state(dom)
    cs = S._c()
    _load().orc_sources(ctypes.byref(dom._c), _cgeom(geom), ctypes.byref(_cstate(U)), ctypes.byref(cs),
                        ctypes.byref(_cstate(dU)))
    return dU


def stage(dom, geom, tabs, Usrc, Ubase, dt, src: Sources | None = None):
    """Uout = R[Ubase + dt * (dU(Usrc) + S(Usrc))] on all four grids (S: the
    sources, none when src is None)."""
    lib = _load()
    _check_state(dom, Usrc)
    _check_state(dom, Ubase)
    out = empty_state(dom)
    scratch = empty_state(dom)
    cw = (_Wsrd * 4)()
    for g in range(4):
        T = tabs[g]
        cw[g] = _Wsrd(*(_ptr(T[k]) for k in ("code", "nnb", "kappa", "omega", "vhat", "xhat")))
    cs = None
    if src is not None:
        assert src.rho0.shape == (dom.nz,) and src.rt0.shape == (dom.nz,)
        cs = src._c()
    lib.orc_stage(ctypes.byref(dom._c), _cgeom(geom), cw, ctypes.byref(_cstate(Usrc)), ctypes.byref(_cstate(Ubase)),
                  float(dt), ctypes.byref(_cstate(out)), ctypes.byref(_cstate(scratch)),
                  ctypes.byref(cs) if cs is not None else None)
    return out


def step(dom, geom, tabs, U, dt, nsteps=1, stages=1, src: Sources | None = None):
    """nsteps steps of Algorithm 1 (stages = 1 or 3), with the sources src
    when given."""
    U = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in U.items()}
    for _ in range(int(nsteps)):
        if stages == 1:
            U = stage(dom, geom, tabs, U, U, dt, src)
        elif stages == 3:
            U1 = stage(dom, geom, tabs, U, U, dt / 3.0, src)
            U2 = stage(dom, geom, tabs, U1, U, dt / 2.0, src)
            U = stage(dom, geom, tabs, U2, U, dt, src)
        else:
            raise ValueError("stages must be 1 or 3")
    return U


def coarse_domain(fine: Domain, h_coarse=None) -> Domain:
    """The coarse level of a refinement ratio 2 over the same domain (Sec.
    4.3): NX/2 x NY/2 x nz/2 cells; its nodal heights default to every other
    fine node (they serve only as a record: the coarse geometry comes from
    ``coarsen``)."""
    assert fine.NX % 2 == 0 and fine.NY % 2 == 0 and fine.nz % 2 == 0
    h = fine.h[::2, ::2] if h_coarse is None else h_coarse
    return Domain(fine.NX // 2, fine.NY // 2, fine.nz // 2, fine.Lx, fine.Ly, fine.Lz, np.ascontiguousarray(h))


def coarsen(fine: Domain, geom: dict, coarse: Domain) -> dict:
    """Geometry of the four grids of the coarse level, merged from the fine
    level's cells (Sec. 4.3; section 6 of eb_oracle.c)."""
    lib = _load()
    fg = _cgeom(geom)
    out = {}
    for g in range(4):
        s = coarse.shape(g)
        G = dict(alpha=np.zeros(s), cent=np.zeros((3,) + s), beta=np.zeros((3,) + s),
                 fcent=np.zeros((6,) + s), aeb=np.zeros(s), nrm=np.zeros((3,) + s),
                 ebc=np.zeros((3,) + s), ebv=np.zeros((3,) + s), flag=np.zeros(s, np.uint8))
        cg = _Geom(*(_ptr(G[k]) for k in ("alpha", "cent", "beta", "fcent", "aeb", "nrm", "ebc", "ebv", "flag")))
        if lib.orc_coarsen(ctypes.byref(fine._c), fg, ctypes.byref(coarse._c), g, ctypes.byref(cg)) != 0:
            raise ValueError("coarsen: the coarse level must halve every fine dimension over the whole domain")
        out[g] = G
    return out


def restrict(fine: Domain, geom: dict, Uf: dict, coarse: Domain, Uc: dict, cols=None) -> dict:
    """The fine state restricted to the coarse level (Sec. 4.3): volume-
    weighted cell-centred fields, area-weighted face fields; coarse CVs with
    no fine fluid or open area keep their values from Uc.  ``cols``: the
    global fine columns (x_lo, x_hi), both even, whose coarse columns are
    restricted (default all); the fine domain may be a window holding them."""
    _check_state(fine, Uf)
    _check_state(coarse, Uc)
    lo, hi = (0, fine.NX) if cols is None else (int(cols[0]), int(cols[1]))
    out = {k: np.ascontiguousarray(Uc[k], dtype=np.float64).copy() for k in FIELDS}
    if _load().orc_restrict(ctypes.byref(fine._c), _cgeom(geom), ctypes.byref(_cstate(Uf)), ctypes.byref(coarse._c),
                            ctypes.byref(_cstate(out)), lo, hi) != 0:
        raise ValueError("restrict: the coarse level must halve every fine dimension, cols even")
    return out


def prolong(coarse: Domain, Uc: dict, fine: Domain, Uf: dict, owned) -> dict:
    """The coarse state prolonged onto the fine window outside its owned
    global fine columns (x_lo, x_hi) (Sec. 4.3: boundary values of a refined
    patch); returns a copy of Uf with those columns filled."""
    _check_state(coarse, Uc)
    _check_state(fine, Uf)
    out = {k: np.ascontiguousarray(Uf[k], dtype=np.float64).copy() for k in FIELDS}
    if _load().orc_prolong(ctypes.byref(coarse._c), ctypes.byref(_cstate(Uc)), ctypes.byref(fine._c),
                           ctypes.byref(_cstate(out)), int(owned[0]), int(owned[1])) != 0:
        raise ValueError("prolong: the coarse level must halve every fine dimension")
    return out


def set_threads(n: int) -> None:
    """OpenMP thread count of later oracle calls (no effect without OpenMP)."""
    try:
        lib = ctypes.CDLL("libgomp.so.1")
        lib.omp_set_num_threads(int(n))
    except OSError:
        pass
