"""Python binding of the C ABI in ``include/eb.h`` (ctypes; argument
marshalling only).  Every step of the method runs in the CUDA library
``libeb.so``; there is no fallback: if the library is missing or no CUDA
device is present, the calls raise.

Tensors are torch CUDA tensors (torch is used for device memory and streams
only).  State fields are dicts with keys ``rho, rhotheta, rhou, rhov, rhow``
shaped (nz, ny, nx) -- (nz+1, ny, nx) for ``rhow`` -- of dtype float64
(``precision="f64"``) or float32 (``precision="mixed"``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")
FIELD_GRID = {"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}
EXPORT_FIELDS = ("alpha", "cent_x", "cent_y", "cent_z", "beta_x", "beta_y", "beta_z", "fcent_x1", "fcent_x2",
                 "fcent_y1", "fcent_y2", "fcent_z1", "fcent_z2", "aeb", "nrm_x", "nrm_y", "nrm_z", "ebc_x",
                 "ebc_y", "ebc_z", "flag", "code", "nnb", "kappa", "omega", "vhat", "xhat_x", "xhat_y", "xhat_z")
STATUS = {0: "EB_OK", 1: "EB_ERR_INVALID_ARG", 2: "EB_ERR_CUDA", 3: "EB_ERR_OOM", 4: "EB_ERR_NUMERIC",
          5: "EB_ERR_TIMEOUT", 6: "EB_ERR_STATE"}
EXPORTED_SYMBOLS = ("eb_geom_build", "eb_geom_destroy", "eb_geom_info", "eb_geom_export", "eb_flux_div", "eb_wsrd",
                    "eb_wsrd_noalloc", "eb_step", "eb_step_profile", "eb_sync_status", "eb_last_error", "eb_version",
                    "eb_ensemble_create", "eb_ensemble_set_state", "eb_ensemble_get_state", "eb_ensemble_step",
                    "eb_ensemble_tune", "eb_ensemble_destroy", "eb_project", "eb_anelastic_step",
                    "eb_unet_num_params", "eb_unet_create", "eb_unet_set_params", "eb_unet_get_params",
                    "eb_unet_forward", "eb_unet_gradient", "eb_unet_train_step", "eb_unet_destroy",
                    "eb_unet_sync_status", "eb_unet_inject_wait_fault", "eb_project_sample", "eb_project_warm",
                    "eb_geom_tune",
                    "eb_geom_set_slab_levels", "eb_geom_set_bulk_priority", "eb_project_set_preconditioner",
                    "eb_geom_set_wind_reference", "eb_fma_peak", "eb_ensemble_info",
                    "eb_ensemble_inject_barrier_fault", "eb_ensemble_set_schedule", "eb_geom_set_sources",
                    "eb_geom_build_coarse", "eb_restrict", "eb_prolong", "eb_geom_set_tile_rows")


class EbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("Lx", ctypes.c_double),
                ("Ly", ctypes.c_double), ("Lz", ctypes.c_double), ("v_target_frac", ctypes.c_double)]


class _State(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in FIELDS]


class GeomInfo(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("cvs", ctypes.c_int64 * 4), ("band_records", ctypes.c_int64 * 4),
                ("small_cvs", ctypes.c_int64 * 4), ("affected_cvs", ctypes.c_int64 * 4),
                ("band_cvs", ctypes.c_int64 * 4), ("band_faces", ctypes.c_int64 * 4),
                ("tiny_cvs", ctypes.c_int64 * 4), ("fast_cells", ctypes.c_int64),
                ("min_alpha", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("slab_levels", ctypes.c_int64),
                ("bulk_high_priority", ctypes.c_int64), ("wsrd_beside_bulk", ctypes.c_int64),
                ("tile_rows", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


_lib = None


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libeb.so (built by ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is missing: run paper_2604_11959_gb300.build.build() first")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, V, I, D = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.eb_geom_build.argtypes = [P(_Desc), V, I, V, V, V, P(V)]
    lib.eb_geom_destroy.argtypes = [V]
    lib.eb_geom_info.argtypes = [V, P(GeomInfo)]
    lib.eb_geom_export.argtypes = [V, I, I, V, V]
    lib.eb_flux_div.argtypes = [V, P(_State), P(_State), V]
    lib.eb_wsrd.argtypes = [V, I, V, V, V]
    lib.eb_wsrd_noalloc.argtypes = [V, I, V, V, V]
    lib.eb_step.argtypes = [V, P(_State), P(_State), D, I, I, V]
    lib.eb_step_profile.argtypes = [V, P(_State), P(_State), D, V, P(ctypes.c_float)]
    lib.eb_sync_status.argtypes = [V, V]
    lib.eb_ensemble_create.argtypes = [P(V), I, P(V)]
    lib.eb_ensemble_set_state.argtypes = [V, I, P(_State), V]
    lib.eb_ensemble_get_state.argtypes = [V, I, P(_State), V]
    lib.eb_ensemble_step.argtypes = [V, P(D), I, V]
    lib.eb_ensemble_tune.argtypes = [V, P(D), I, P(I), V]
    lib.eb_ensemble_destroy.argtypes = [V]
    lib.eb_project.argtypes = [V, P(_State), D, D, I, V, V, P(I), P(D), V]
    lib.eb_anelastic_step.argtypes = [V, P(_State), P(_State), D, I, D, I, P(I), V]
    F, L = ctypes.c_float, ctypes.c_int64
    lib.eb_unet_num_params.restype = L
    lib.eb_unet_create.argtypes = [I, I, I, P(V)]
    lib.eb_unet_set_params.argtypes = [V, V, L]
    lib.eb_unet_get_params.argtypes = [V, V, L]
    lib.eb_unet_forward.argtypes = [V, V, V, V]
    lib.eb_unet_gradient.argtypes = [V, V, V, V, P(F), V, V]
    lib.eb_unet_train_step.argtypes = [V, V, V, V, F, P(F), V]
    lib.eb_unet_destroy.argtypes = [V]
    lib.eb_unet_sync_status.argtypes = [V]
    lib.eb_unet_inject_wait_fault.argtypes = [V]
    lib.eb_project_sample.argtypes = [V, P(_State), D, D, I, D, V, V, V, P(I), V]
    lib.eb_project_warm.argtypes = [V, V, P(_State), D, D, I, D, P(I), P(D), V]
    lib.eb_geom_tune.argtypes = [V, P(_State), D, I, P(I), V]
    lib.eb_geom_set_slab_levels.argtypes = [V, I]
    lib.eb_geom_set_bulk_priority.argtypes = [V, I]
    lib.eb_project_set_preconditioner.argtypes = [V, I]
    lib.eb_geom_set_wind_reference.argtypes = [V, V, V, V]
    lib.eb_geom_set_sources.argtypes = [V, I]
    lib.eb_geom_set_tile_rows.argtypes = [V, I]
    lib.eb_geom_build_coarse.argtypes = [V, V, V, V, V]
    lib.eb_restrict.argtypes = [V, V, V, V, I, I, I, V]
    lib.eb_prolong.argtypes = [V, V, V, V, I, I, I, V]
    lib.eb_fma_peak.argtypes = [I, P(D), V]
    lib.eb_ensemble_info.argtypes = [V, P(I)]
    lib.eb_ensemble_inject_barrier_fault.argtypes = [V, I]
    lib.eb_ensemble_set_schedule.argtypes = [V, I]
    lib.eb_last_error.restype = ctypes.c_char_p
    lib.eb_version.restype = I
    for name in ("eb_geom_build", "eb_geom_destroy", "eb_geom_info", "eb_geom_export", "eb_flux_div", "eb_wsrd",
                 "eb_wsrd_noalloc", "eb_step", "eb_step_profile", "eb_sync_status", "eb_ensemble_create",
                 "eb_ensemble_set_state", "eb_ensemble_get_state", "eb_ensemble_step", "eb_ensemble_tune",
                 "eb_ensemble_destroy", "eb_project", "eb_anelastic_step", "eb_unet_create", "eb_unet_set_params",
                 "eb_unet_get_params", "eb_unet_forward", "eb_unet_gradient", "eb_unet_train_step",
                 "eb_unet_destroy", "eb_unet_sync_status", "eb_unet_inject_wait_fault", "eb_project_sample",
                 "eb_project_warm", "eb_geom_tune",
                 "eb_geom_set_slab_levels", "eb_geom_set_bulk_priority", "eb_project_set_preconditioner",
                 "eb_geom_set_wind_reference", "eb_fma_peak", "eb_ensemble_info",
                 "eb_ensemble_inject_barrier_fault", "eb_ensemble_set_schedule", "eb_geom_set_sources",
                 "eb_geom_build_coarse", "eb_restrict", "eb_prolong", "eb_geom_set_tile_rows"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(code: int):
    if code != 0:
        raise EbError(code, load().eb_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require_cuda(t: torch.Tensor, dtype, shape, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Geometry:
    """Handle of the geometry of all four grids and the redistribution tables
    (``eb_geom_build``)."""

    def __init__(self, nx, ny, nz, Lx, Ly, Lz, h_nodes: torch.Tensor, precision: str = "f64", ref_rho=None,
                 ref_rhotheta=None, v_target_frac: float = 0.5, stream=None, ref_rhou=None, ref_rhov=None):
        lib = load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.Lx, self.Ly, self.Lz = float(Lx), float(Ly), float(Lz)
        self.precision = precision
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        prec = {"f64": 0, "mixed": 1}[precision]
        _require_cuda(h_nodes, torch.float64, (self.ny + 1, self.nx + 1), "h_nodes")
        refs = [None, None]
        for q, r in enumerate((ref_rho, ref_rhotheta)):
            if r is not None:
                _require_cuda(r, torch.float64, (self.nz,), "reference profile")
                refs[q] = r
        self._keep = (h_nodes, refs)
        desc = _Desc(self.nx, self.ny, self.nz, self.Lx, self.Ly, self.Lz, float(v_target_frac))
        handle = ctypes.c_void_p()
        _check(lib.eb_geom_build(ctypes.byref(desc), h_nodes.data_ptr(), prec,
                                 refs[0].data_ptr() if refs[0] is not None else None,
                                 refs[1].data_ptr() if refs[1] is not None else None, _stream(stream),
                                 ctypes.byref(handle)))
        self._h = handle
        if ref_rhou is not None or ref_rhov is not None:
            self.set_wind_reference(ref_rhou, ref_rhov, stream)

    def set_wind_reference(self, ref_rhou=None, ref_rhov=None, stream=None):
        """Background momentum profiles (``eb_geom_set_wind_reference``):
        CUDA float64 tensors of nz values or None (zero).  Later rho*u and
        rho*v states hold values minus the profile."""
        for r in (ref_rhou, ref_rhov):
            if r is not None:
                _require_cuda(r, torch.float64, (self.nz,), "momentum profile")
        _check(load().eb_geom_set_wind_reference(self.handle, ref_rhou.data_ptr() if ref_rhou is not None else None,
                                                 ref_rhov.data_ptr() if ref_rhov is not None else None,
                                                 _stream(stream)))
        self._wind = (ref_rhou, ref_rhov)

    def set_sources(self, pressure: bool = True, buoyancy: bool = True):
        """Sources of the compressible system that eb_step adds to every stage
        (``eb_geom_set_sources``): the perturbation pressure gradient from the
        equation of state and the buoyancy; both False switches them off."""
        _check(load().eb_geom_set_sources(self.handle, (1 if pressure else 0) | (2 if buoyancy else 0)))

    def coarse(self, ref_rho=None, ref_rhotheta=None, stream=None) -> "Geometry":
        """The coarse level of a refinement ratio 2 (``eb_geom_build_coarse``):
        nx/2 x ny/2 x nz/2 cells, geometry merged from this handle's cells;
        reference profiles of nz/2 levels (CUDA float64) or None."""
        refs = [None, None]
        for q, r in enumerate((ref_rho, ref_rhotheta)):
            if r is not None:
                _require_cuda(r, torch.float64, (self.nz // 2,), "reference profile")
                refs[q] = r
        handle = ctypes.c_void_p()
        _check(load().eb_geom_build_coarse(self.handle, refs[0].data_ptr() if refs[0] is not None else None,
                                           refs[1].data_ptr() if refs[1] is not None else None, _stream(stream),
                                           ctypes.byref(handle)))
        g = Geometry.__new__(Geometry)
        g.nx, g.ny, g.nz = self.nx // 2, self.ny // 2, self.nz // 2
        g.Lx, g.Ly, g.Lz = self.Lx, self.Ly, self.Lz
        g.precision, g.dtype = self.precision, self.dtype
        g._keep = (None, refs)
        g._h = handle
        return g

    def close(self):
        if getattr(self, "_h", None):
            load().eb_geom_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("geometry handle was closed")
        return self._h

    def shape(self, field_or_grid):
        g = FIELD_GRID[field_or_grid] if isinstance(field_or_grid, str) else int(field_or_grid)
        return (self.nz + (1 if g == 3 else 0), self.ny, self.nx)

    def info(self) -> dict:
        inf = GeomInfo()
        _check(load().eb_geom_info(self.handle, ctypes.byref(inf)))
        return inf.as_dict()

    def export(self, grid: int, field: str, stream=None) -> torch.Tensor:
        out = torch.empty(self.shape(int(grid)), dtype=torch.float64, device="cuda")
        _check(load().eb_geom_export(self.handle, int(grid), EXPORT_FIELDS.index(field), out.data_ptr(),
                                     _stream(stream)))
        return out

    def empty_state(self) -> dict:
        return {f: torch.empty(self.shape(f), dtype=self.dtype, device="cuda") for f in FIELDS}

    def packed_state(self, device: str = "cuda", pin: bool = False):
        """One allocation holding all five fields (each starting on a 256-byte
        boundary), returned as (flat tensor, dict of per-field views): a whole
        state moves between host and device with one copy of the flat tensor."""
        es = torch.empty((), dtype=self.dtype).element_size()
        align = 256 // es
        offs, n = {}, 0
        for f in FIELDS:
            offs[f] = n
            cnt = int(np.prod(self.shape(f)))
            n += (cnt + align - 1) // align * align
        flat = torch.empty(n, dtype=self.dtype, device=device)
        if pin:
            flat = flat.pin_memory()
        views = {f: flat[offs[f]:offs[f] + int(np.prod(self.shape(f)))].view(self.shape(f)) for f in FIELDS}
        return flat, views

    def _cstate(self, U: dict) -> _State:
        for f in FIELDS:
            _require_cuda(U[f], self.dtype, self.shape(f), f)
        return _State(*(U[f].data_ptr() for f in FIELDS))


def flux_div(geom: Geometry, U: dict, out: dict | None = None, stream=None) -> dict:
    """dU of every field (``eb_flux_div``)."""
    out = out if out is not None else geom.empty_state()
    _check(load().eb_flux_div(geom.handle, ctypes.byref(geom._cstate(U)), ctypes.byref(geom._cstate(out)),
                              _stream(stream)))
    return out


def wsrd(geom: Geometry, field: str, Uhat: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Redistribution of one field (``eb_wsrd``); ``out`` may be ``Uhat``."""
    _require_cuda(Uhat, geom.dtype, geom.shape(field), field)
    out = out if out is not None else torch.empty_like(Uhat)
    _require_cuda(out, geom.dtype, geom.shape(field), "out")
    _check(load().eb_wsrd(geom.handle, FIELDS.index(field), Uhat.data_ptr(), out.data_ptr(), _stream(stream)))
    return out


def wsrd_noalloc(geom: Geometry, field: str, Uhat: torch.Tensor, out: torch.Tensor, stream=None):
    """Redistribution of one field through ``eb_wsrd_noalloc``: scratch from
    the library's fixed device block, nothing allocated.  ``out`` is required
    (it may be ``Uhat``) so that this call allocates nothing either."""
    _require_cuda(Uhat, geom.dtype, geom.shape(field), field)
    _require_cuda(out, geom.dtype, geom.shape(field), "out")
    _check(load().eb_wsrd_noalloc(geom.handle, FIELDS.index(field), Uhat.data_ptr(), out.data_ptr(),
                                  _stream(stream)))
    return out


def step(geom: Geometry, Un: dict, dt: float, nsteps: int = 1, stages: int = 1, out: dict | None = None,
         stream=None) -> dict:
    """nsteps steps of Algorithm 1 (``eb_step``)."""
    out = out if out is not None else geom.empty_state()
    _check(load().eb_step(geom.handle, ctypes.byref(geom._cstate(Un)), ctypes.byref(geom._cstate(out)), float(dt),
                          int(nsteps), int(stages), _stream(stream)))
    return out


def step_profile(geom: Geometry, Un: dict, out: dict, dt: float, stream=None):
    """One forward-Euler step with per-phase event times (``eb_step_profile``):
    returns milliseconds of (bulk flux kernel, near-EB flux kernel,
    redistribution, whole step)."""
    ms = (ctypes.c_float * 4)()
    _check(load().eb_step_profile(geom.handle, ctypes.byref(geom._cstate(Un)), ctypes.byref(geom._cstate(out)),
                                  float(dt), _stream(stream), ms))
    return tuple(float(v) for v in ms)


def project(geom: Geometry, U: dict, dt: float, rtol: float = 1e-10, maxit: int = 100000, phi0=None,
            phi=None, stream=None):
    """Projection of the face momenta of U in place (``eb_project``).
    Returns (iterations, relative residual); phi (if given) receives the
    solution, phi0 (if given) is the initial guess."""
    shape = geom.shape(0)
    for name, t in (("phi0", phi0), ("phi", phi)):
        if t is not None:
            _require_cuda(t, torch.float64, shape, name)
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    _check(load().eb_project(geom.handle, ctypes.byref(geom._cstate(U)), float(dt), float(rtol), int(maxit),
                             phi0.data_ptr() if phi0 is not None else None,
                             phi.data_ptr() if phi is not None else None, ctypes.byref(it), ctypes.byref(res),
                             _stream(stream)))
    return it.value, res.value


def anelastic_step(geom: Geometry, Un: dict, dt: float, nsteps: int = 1, rtol: float = 1e-10,
                   maxit: int = 100000, out: dict | None = None, stream=None):
    """nsteps anelastic steps (``eb_anelastic_step``); returns (state,
    iterations of every projection)."""
    out = out if out is not None else geom.empty_state()
    its = (ctypes.c_int * (2 * int(nsteps)))()
    _check(load().eb_anelastic_step(geom.handle, ctypes.byref(geom._cstate(Un)), ctypes.byref(geom._cstate(out)),
                                    float(dt), int(nsteps), float(rtol), int(maxit), its, _stream(stream)))
    return out, list(its)


def tune(geom: Geometry, U: dict, dt: float, reps: int = 5, stream=None) -> int:
    """Autotune the bulk kernel's slab height on U (``eb_geom_tune``);
    returns the chosen height (0 = automatic)."""
    best = ctypes.c_int(0)
    _check(load().eb_geom_tune(geom.handle, ctypes.byref(geom._cstate(U)), float(dt), int(reps), ctypes.byref(best),
                               _stream(stream)))
    return best.value


PRECONDITIONERS = {"jacobi": 0, "mg": 1}


def set_preconditioner(geom: Geometry, kind: str) -> None:
    """Preconditioner of the projection's conjugate gradients for this handle
    (``eb_project_set_preconditioner``): "jacobi" (default) or "mg"."""
    if kind not in PRECONDITIONERS:
        raise ValueError(f"unknown preconditioner {kind!r}")
    _check(load().eb_project_set_preconditioner(geom.handle, PRECONDITIONERS[kind]))


def set_bulk_priority(geom: Geometry, high: bool) -> None:
    """Run the bulk kernel on a high-priority stream beside the near-EB
    kernels, or on the caller's stream (``eb_geom_set_bulk_priority``)."""
    _check(load().eb_geom_set_bulk_priority(geom.handle, 1 if high else 0))


def set_tile_rows(geom: Geometry, rows: int) -> None:
    """Rows of the bulk kernel's tiles, 16 or (mixed path) 14
    (``eb_geom_set_tile_rows``)."""
    _check(load().eb_geom_set_tile_rows(geom.handle, int(rows)))


def set_slab_levels(geom: Geometry, levels: int) -> None:
    """Set the bulk kernel's slab height (``eb_geom_set_slab_levels``)."""
    _check(load().eb_geom_set_slab_levels(geom.handle, int(levels)))


def restrict(fine: Geometry, coarse: Geometry, Uf: dict, Uc: dict, fine_x0: int = 0, cols=None, stream=None) -> dict:
    """A fine state restricted onto the coarse level in place of Uc
    (``eb_restrict``): volume-weighted cell-centred fields, area-weighted face
    fields; coarse CVs without fine fluid keep their values.  The fine handle
    may be an x-window of the fine level starting at global fine column
    fine_x0; ``cols`` = (lo, hi) local fine columns to restrict (default
    all).  Returns Uc."""
    lo, hi = (0, fine.nx) if cols is None else (int(cols[0]), int(cols[1]))
    _check(load().eb_restrict(fine.handle, coarse.handle, ctypes.byref(fine._cstate(Uf)),
                              ctypes.byref(coarse._cstate(Uc)), int(fine_x0), lo, hi, _stream(stream)))
    return Uc


def prolong(coarse: Geometry, Uc: dict, fine: Geometry, Uf: dict, fine_x0: int = 0, owned=(0, 0),
            stream=None) -> dict:
    """The coarse state prolonged onto every column of the fine handle
    outside its local columns ``owned`` = (lo, hi) (``eb_prolong``: boundary
    values of a refined patch), in place of Uf.  Returns Uf."""
    _check(load().eb_prolong(coarse.handle, ctypes.byref(coarse._cstate(Uc)), fine.handle,
                             ctypes.byref(fine._cstate(Uf)), int(fine_x0), int(owned[0]), int(owned[1]),
                             _stream(stream)))
    return Uf


def fma_peak(kind: str, stream=None) -> float:
    """Measured fused multiply-add throughput of this GPU in GFLOP/s
    (``eb_fma_peak``): kind "f64" (DFMA), "f32" (FFMA) or "f32x2" (packed
    FFMA2); an FMA counts as two flops."""
    out = ctypes.c_double(0.0)
    _check(load().eb_fma_peak({"f64": 0, "f32": 1, "f32x2": 2}[kind], ctypes.byref(out), _stream(stream)))
    return out.value


def sync_status(geom: Geometry, stream=None) -> None:
    """Raise EbError if a kernel latched a device-side error (``eb_sync_status``)."""
    _check(load().eb_sync_status(geom.handle, _stream(stream)))


# fields that carry a per-level profile, in the order of a ``refs`` tuple
REF_FIELDS = ("rho", "rhotheta", "rhou", "rhov")


def host_state(U: dict, precision: str, refs=None, pin: bool = True) -> dict:
    """CPU tensors of a state given as numpy full values: float64 or float32,
    each field minus its per-level profile when ``refs`` gives one: ``refs =
    (rho0, rho0*theta0)`` or ``(rho0, rho0*theta0, ref_rhou, ref_rhov)`` (the
    last two as set with ``Geometry.set_wind_reference``; None entries are
    zero).  Pinned for asynchronous copies."""
    import numpy as np
    dt = torch.float64 if precision == "f64" else torch.float32
    out = {}
    for f in FIELDS:
        a = U[f]
        q = REF_FIELDS.index(f) if f in REF_FIELDS else None
        if refs is not None and q is not None and q < len(refs) and refs[q] is not None:
            a = a - np.asarray(refs[q])[:, None, None]
        t = torch.from_numpy(np.ascontiguousarray(a)).to(dt)
        out[f] = t.pin_memory() if pin else t
    return out


def device_state(U: dict, precision: str, refs=None) -> dict:
    """Like host_state, on the current CUDA device."""
    return {f: t.cuda() for f, t in host_state(U, precision, refs, pin=False).items()}


def full_values(U: dict, refs=None) -> dict:
    """numpy float64 full values of a state (torch tensors, device or host):
    the inverse of host_state / device_state, profiles added back."""
    out = {}
    for f in FIELDS:
        a = U[f].double().cpu().numpy()
        q = REF_FIELDS.index(f) if f in REF_FIELDS else None
        if refs is not None and q is not None and q < len(refs) and refs[q] is not None:
            a = a + np.asarray(refs[q])[:, None, None]
        out[f] = a
    return out


class Ensemble:
    """Independent geometry handles advanced together (``eb_ensemble_*``):
    one CUDA-graph launch per step of every member, slab heights of the bulk
    kernel's tiles chosen by ``tune``.  The ensemble does not own the
    members; close it before them."""

    def __init__(self, members):
        lib = load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.handle.value for m in self.members])
        h = ctypes.c_void_p()
        _check(lib.eb_ensemble_create(arr, len(self.members), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("ensemble is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().eb_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dt(self, dt):
        dt = [float(x) for x in dt]
        if len(dt) != len(self.members):
            raise ValueError("one dt per member")
        return (ctypes.c_double * len(dt))(*dt)

    def set_state(self, q: int, U: dict, stream=None):
        g = self.members[q]
        for f in FIELDS:
            _require_cuda(U[f], g.dtype, g.shape(f), f)
        _check(load().eb_ensemble_set_state(self.handle, q, ctypes.byref(g._cstate(U)), _stream(stream)))

    def get_state(self, q: int, out: dict | None = None, stream=None) -> dict:
        g = self.members[q]
        out = out if out is not None else g.empty_state()
        _check(load().eb_ensemble_get_state(self.handle, q, ctypes.byref(g._cstate(out)), _stream(stream)))
        return out

    def step(self, dt, nsteps: int = 1, stream=None):
        _check(load().eb_ensemble_step(self.handle, self._dt(dt), int(nsteps), _stream(stream)))

    def tune(self, dt, reps: int = 3, stream=None) -> int:
        best = ctypes.c_int(0)
        _check(load().eb_ensemble_tune(self.handle, self._dt(dt), int(reps), ctypes.byref(best), _stream(stream)))
        return best.value

    def info(self) -> dict:
        """Launch figures of the persistent step kernel (``eb_ensemble_info``)."""
        v = (ctypes.c_int * 6)()
        _check(load().eb_ensemble_info(self.handle, v))
        return {"ctas": v[0], "units": v[1], "registers": v[2], "static_smem": v[3], "local_bytes": v[4],
                "schedule": ("persistent", "branches")[v[5]]}

    def set_schedule(self, schedule: str):
        """"persistent" (one cooperative launch per step) or "branches" (each
        member's kernels side by side); ``eb_ensemble_set_schedule``."""
        _check(load().eb_ensemble_set_schedule(self.handle, {"persistent": 0, "branches": 1}[schedule]))

    def inject_barrier_fault(self, cta: int):
        """Failure test: CTA ``cta`` of later steps skips the first barrier
        (-1 restores normal steps); ``eb_ensemble_inject_barrier_fault``."""
        _check(load().eb_ensemble_inject_barrier_fault(self.handle, int(cta)))


class UNet:
    """The warm-start network of the projection (``eb_unet_*``), sized for
    one grid.  Parameters are a flat float32 numpy vector."""

    def __init__(self, nx: int, ny: int, nz: int):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.eb_unet_create(int(nx), int(ny), int(nz), ctypes.byref(h)))
        self._h = h
        self.shape = (int(nz), int(ny), int(nx))
        self.n = int(lib.eb_unet_num_params())

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("network is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().eb_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.n:
            raise ValueError("wrong parameter count")
        _check(load().eb_unet_set_params(self.handle, p.ctypes.data, self.n))

    def get_params(self):
        import numpy as np
        p = np.zeros(self.n, dtype=np.float32)
        _check(load().eb_unet_get_params(self.handle, p.ctypes.data, self.n))
        return p

    def _need(self, t, ch, name):
        _require_cuda(t, torch.float32, (ch,) + self.shape if ch > 1 else self.shape, name)

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        self._need(x, 2, "input")
        out = out if out is not None else torch.empty(self.shape, dtype=torch.float32, device="cuda")
        self._need(out, 1, "out")
        _check(load().eb_unet_forward(self.handle, x.data_ptr(), out.data_ptr(), _stream(stream)))
        return out

    def gradient(self, x, target, mask, stream=None):
        """(loss, flat gradient as numpy float32)."""
        import numpy as np
        for t, ch, nm in ((x, 2, "input"), (target, 1, "target"), (mask, 1, "mask")):
            self._need(t, ch, nm)
        loss = ctypes.c_float(0.0)
        g = np.zeros(self.n, dtype=np.float32)
        _check(load().eb_unet_gradient(self.handle, x.data_ptr(), target.data_ptr(), mask.data_ptr(),
                                       ctypes.byref(loss), g.ctypes.data, _stream(stream)))
        return loss.value, g

    def sync_status(self):
        """Raise EbError (EB_ERR_TIMEOUT) if a convolution's bounded wait
        expired since the last check."""
        _check(load().eb_unet_sync_status(self.handle))

    def inject_wait_fault(self):
        """The failure test: the next convolution never signals its products'
        completion (``eb_unet_inject_wait_fault``)."""
        _check(load().eb_unet_inject_wait_fault(self.handle))

    def train_step(self, x, target, mask, lr: float, want_loss: bool = False, stream=None):
        for t, ch, nm in ((x, 2, "input"), (target, 1, "target"), (mask, 1, "mask")):
            self._need(t, ch, nm)
        loss = ctypes.c_float(0.0)
        _check(load().eb_unet_train_step(self.handle, x.data_ptr(), target.data_ptr(), mask.data_ptr(),
                                         float(lr), ctypes.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None


def project_sample(geom: Geometry, U: dict, dt: float, scale: float, rtol: float = 1e-10, maxit: int = 100000,
                   stream=None):
    """A training sample (input, target, mask, iterations) from the momenta
    of U (``eb_project_sample``)."""
    shape = geom.shape(0)
    x = torch.empty((2,) + shape, dtype=torch.float32, device="cuda")
    t = torch.empty(shape, dtype=torch.float32, device="cuda")
    m = torch.empty(shape, dtype=torch.float32, device="cuda")
    it = ctypes.c_int(0)
    _check(load().eb_project_sample(geom.handle, ctypes.byref(geom._cstate(U)), float(dt), float(rtol), int(maxit),
                                    float(scale), x.data_ptr(), t.data_ptr(), m.data_ptr(), ctypes.byref(it),
                                    _stream(stream)))
    return x, t, m, it.value


def project_warm(geom: Geometry, net: UNet, U: dict, dt: float, scale: float, rtol: float = 1e-10,
                 maxit: int = 100000, stream=None):
    """Projection of U's momenta in place from the network's initial guess
    (``eb_project_warm``); returns (iterations, relative residual)."""
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    _check(load().eb_project_warm(geom.handle, net.handle, ctypes.byref(geom._cstate(U)), float(dt), float(rtol),
                                  int(maxit), float(scale), ctypes.byref(it), ctypes.byref(res), _stream(stream)))
    return it.value, res.value
