"""Python binding of libfld.so (argument marshalling only).

Every function here has the name of the C entry point it calls (see
include/fld.h) and forwards plain pointers and sizes: device tensors are
passed as ``torch.Tensor`` (CUDA, float64, contiguous), host arrays for
``fld_step_host`` as numpy float64 arrays.  All arithmetic of the step runs
in the library's CUDA kernels; if the library cannot be built or loaded the
import of the first call raises -- there is no other implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

FLD_OK, FLD_EINVAL, FLD_ENOMEM, FLD_ENOCONV, FLD_ENONFINITE, FLD_ETIMEOUT, FLD_ECUDA = range(7)
STATUS_NAMES = {0: "FLD_OK", 1: "FLD_EINVAL", 2: "FLD_ENOMEM", 3: "FLD_ENOCONV",
                4: "FLD_ENONFINITE", 5: "FLD_ETIMEOUT", 6: "FLD_ECUDA"}


class FldError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


FLD_BC_ZERO_GRADIENT, FLD_BC_PERIODIC, FLD_BC_DIRICHLET, FLD_BC_OUTFLOW = range(4)


class fld_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3), ("bc_value", ctypes.c_double * 6)]


class fld_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("c", ctypes.c_double), ("L_unit", ctypes.c_double),
                ("dmax_coef", ctypes.c_double), ("rmin_coef", ctypes.c_double),
                ("sigma", ctypes.c_double), ("adot_over_a", ctypes.c_double),
                ("hnu", ctypes.c_double), ("limiter", ctypes.c_int), ("precision", ctypes.c_int),
                ("smoother", ctypes.c_int), ("jacobi_omega", ctypes.c_double),
                ("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("pre", ctypes.c_int),
                ("post", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("coarse_cap", ctypes.c_int), ("graphs", ctypes.c_int), ("fused_post", ctypes.c_int),
                ("theta", ctypes.c_double), ("scale_factor", ctypes.c_double), ("tail_cells", ctypes.c_int),
                ("paper_order", ctypes.c_int), ("persistent_cells", ctypes.c_int),
                ("precond_bf16", ctypes.c_int)]


class fld_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("balance_abs", ctypes.c_double),
                ("balance_rel", ctypes.c_double), ("emitted", ctypes.c_double),
                ("absorbed", ctypes.c_double), ("floor_added", ctypes.c_double),
                ("rel_change", ctypes.c_double), ("ms", ctypes.c_double), ("outflow", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fld_advance_params(ctypes.Structure):
    _fields_ = [("tau_tol", ctypes.c_double), ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("growth", ctypes.c_double), ("max_substeps", ctypes.c_int)]


class fld_advance_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("substeps", ctypes.c_int), ("retries", ctypes.c_int),
                ("iters", ctypes.c_int), ("t_done", ctypes.c_double), ("dt_next", ctypes.c_double),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FLD_SED_MONO, FLD_SED_BLACKBODY, FLD_SED_POWERLAW = range(3)
FLD_MAX_GROUPS = 16
FLD_SED_NCOEF = 10


class fld_xsec(ctypes.Structure):
    _fields_ = [("nu_threshold", ctypes.c_double), ("sigma0", ctypes.c_double), ("beta", ctypes.c_double),
                ("s", ctypes.c_double)]


class fld_sed(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nu_mono", ctypes.c_double), ("T", ctypes.c_double),
                ("alpha", ctypes.c_double), ("species", fld_xsec * 3)]


class fld_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong),
                ("timed", ctypes.c_longlong), ("ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("timed_bytes", ctypes.c_double)]


_P = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_lib = None
_lock = threading.Lock()

_SIGS = {
    "fld_params_default": ([ctypes.POINTER(fld_params)], ctypes.c_int),
    "fld_footprint_bytes": ([ctypes.POINTER(fld_grid), ctypes.POINTER(fld_params)], ctypes.c_size_t),
    "fld_create": ([ctypes.POINTER(_VP), ctypes.POINTER(fld_grid), ctypes.POINTER(fld_params), _VP],
                   ctypes.c_int),
    "fld_assemble": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "fld_solve": ([_VP, _VP, ctypes.POINTER(fld_info)], ctypes.c_int),
    "fld_step": ([_VP, _VP, _VP, _VP, ctypes.POINTER(fld_info)], ctypes.c_int),
    "fld_step_host": ([_VP, _VP, _VP, _VP, ctypes.POINTER(fld_info)], ctypes.c_int),
    "fld_step_batched": ([ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                          ctypes.POINTER(_VP), ctypes.POINTER(fld_info)], ctypes.c_int),
    "fld_apply": ([_VP, _VP, _VP], ctypes.c_int),
    "fld_vcycle": ([_VP, _VP, _VP], ctypes.c_int),
    "fld_get_system": ([_VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "fld_opacity_update": ([ctypes.c_size_t, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP], ctypes.c_int),
    "fld_levels": ([ctypes.POINTER(fld_grid), ctypes.POINTER(ctypes.c_int), ctypes.c_int], ctypes.c_int),
    "fld_set_dt": ([_VP, ctypes.c_double], ctypes.c_int),
    "fld_set_expansion": ([_VP, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "fld_residual_noalloc": ([ctypes.POINTER(fld_grid)] + [_VP] * 9, ctypes.c_int),
    "fld_advance": ([_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                     ctypes.POINTER(fld_advance_params), ctypes.POINTER(fld_advance_info)], ctypes.c_int),
    "fld_autotune": ([_VP, ctypes.c_int], ctypes.c_int),
    "fld_tuning_size": ([_VP], ctypes.c_int),
    "fld_get_tuning": ([_VP, ctypes.POINTER(ctypes.c_int), ctypes.c_int], ctypes.c_int),
    "fld_set_tuning": ([_VP, ctypes.POINTER(ctypes.c_int), ctypes.c_int], ctypes.c_int),
    "fld_profile": ([_VP, ctypes.c_ulonglong], ctypes.c_int),
    "fld_profile_read": ([_VP, ctypes.POINTER(fld_kernel_stat), ctypes.c_int], ctypes.c_int),
    "fld_sed_default": ([ctypes.POINTER(fld_sed)], ctypes.c_int),
    "fld_sed_integrals": ([ctypes.POINTER(fld_sed), _VP, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "fld_group_fields": ([ctypes.c_size_t, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "fld_photo_rates": ([ctypes.c_size_t, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_double,
                         _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "fld_last_error": ([], ctypes.c_char_p),
    "fld_destroy": ([_VP], None),
}

EXPORTS = tuple(_SIGS)


def lib():
    """Load (building first if needed) the in-tree libfld.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            h = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                f = getattr(h, name)
                f.argtypes = args
                f.restype = res
            _lib = h
    return _lib


def fld_last_error() -> str:
    """The message of the calling thread's last failed call."""
    return lib().fld_last_error().decode()


def _check(st: int, what: str):
    if st != FLD_OK:
        raise FldError(st, f"{what}: {fld_last_error()}")


def _get(o, k, default=None):
    return o.get(k, default) if isinstance(o, dict) else getattr(o, k, default)


def make_grid(g) -> fld_grid:
    """fld_grid of a grid record: n, h, periodic (3 flags) and optionally
    dirichlet (6 flags, x lo, x hi, y lo, ...) with values ebc (6)."""
    n, h, per = _get(g, "n"), _get(g, "h"), _get(g, "periodic")
    dflag = _get(g, "dirichlet") or (False,) * 6
    dval = _get(g, "ebc") or (0.0,) * 6
    lo, hi = [], []
    for a in range(3):
        if per[a]:
            # a Dirichlet flag on a periodic axis is passed on for the
            # library to reject
            lo.append(FLD_BC_PERIODIC)
            hi.append(FLD_BC_DIRICHLET if (dflag[2 * a] or dflag[2 * a + 1]) else FLD_BC_PERIODIC)
        else:
            lo.append(FLD_BC_DIRICHLET if dflag[2 * a] else FLD_BC_ZERO_GRADIENT)
            hi.append(FLD_BC_DIRICHLET if dflag[2 * a + 1] else FLD_BC_ZERO_GRADIENT)
    return fld_grid(int(n[0]), int(n[1]), int(n[2]), float(h[0]), float(h[1]), float(h[2]),
                    (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*hi),
                    (ctypes.c_double * 6)(*[float(v) for v in dval]))


def make_params(p=None, **overrides) -> fld_params:
    """fld_params: the library defaults, then the fields of p (a synth.Params or
    an fld_params) and the keyword overrides."""
    out = fld_params()
    _check(lib().fld_params_default(ctypes.byref(out)), "fld_params_default")
    if p is not None:
        for name, _ in fld_params._fields_:
            v = _get(p, name)
            if v is not None:
                setattr(out, name, type(getattr(out, name))(v))
    for k, v in overrides.items():
        setattr(out, k, type(getattr(out, k))(v))
    return out


def _dptr(t, n=None, what="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{what} must be contiguous float64")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, n, what="array"):
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError(f"{what} must be a C-contiguous float64 numpy array")
    if a.size != n:
        raise ValueError(f"{what} has {a.size} elements, expected {n}")
    return ctypes.c_void_p(a.ctypes.data)


def fld_footprint_bytes(grid, params) -> int:
    """Device bytes a context of this grid and these parameters allocates (0 if
    the pair is invalid); the serving admission uses it."""
    g, p = make_grid(grid), make_params(params)
    return int(lib().fld_footprint_bytes(ctypes.byref(g), ctypes.byref(p)))


def fld_levels(grid) -> List[tuple]:
    """The multigrid level shapes (nx, ny, nz), finest first."""
    g = make_grid(grid)
    dims = (ctypes.c_int * 96)()
    nl = lib().fld_levels(ctypes.byref(g), dims, 32)
    return [tuple(dims[3 * l: 3 * l + 3]) for l in range(nl)]


class Context:
    """Owns one fld_ctx: a grid, parameters, a stream and device buffers."""

    def __init__(self, grid, params=None, stream=None, **overrides):
        import torch
        self.grid = grid
        self._g = make_grid(grid)
        self._p = make_params(params, **overrides)
        self.n = self._g.nx * self._g.ny * self._g.nz
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = _VP()
        _check(lib().fld_create(ctypes.byref(handle), ctypes.byref(self._g), ctypes.byref(self._p),
                                _VP(stream.cuda_stream)), "fld_create")
        self.handle = handle

    @property
    def params(self) -> fld_params:
        return self._p

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().fld_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fld_create(grid, params=None, stream=None, **overrides) -> Context:
    """A context (hierarchy and work buffers on the device) working on stream
    (the current torch stream if None; graphs need a non-default one)."""
    return Context(grid, params, stream, **overrides)


def fld_destroy(ctx: Context):
    """Free the context's device memory (same as ctx.close())."""
    ctx.close()


def fld_assemble(ctx: Context, E, nHI, eta):
    """Assemble the operator and right-hand side of a step from the device
    tensors E, n_HI and eta (FP64, one value per cell)."""
    _check(lib().fld_assemble(ctx.handle, _dptr(E, ctx.n, "E"), _dptr(nHI, ctx.n, "n_HI"),
                              _dptr(eta, ctx.n, "eta")), "fld_assemble")


def fld_solve(ctx: Context, dE, check: bool = True) -> dict:
    """Solve the assembled system into dE; returns the info dict (status,
    iters, outer_iters, rel_res, ...); raises on failure if check."""
    info = fld_info()
    st = lib().fld_solve(ctx.handle, _dptr(dE, ctx.n, "dE"), ctypes.byref(info))
    if check:
        _check(st, "fld_solve")
    d = info.as_dict()
    d["status"] = st
    return d


def fld_step(ctx: Context, E, nHI, eta, check: bool = True) -> dict:
    """One step, E <- max(E + dE, 0) in place on the device; returns the info
    dict with the photon balance; raises on failure if check (E unchanged)."""
    info = fld_info()
    st = lib().fld_step(ctx.handle, _dptr(E, ctx.n, "E"), _dptr(nHI, ctx.n, "n_HI"),
                        _dptr(eta, ctx.n, "eta"), ctypes.byref(info))
    if check:
        _check(st, "fld_step")
    d = info.as_dict()
    d["status"] = st
    return d


def fld_step_host(ctx: Context, E: np.ndarray, nHI: np.ndarray, eta: np.ndarray,
                  check: bool = True) -> dict:
    """fld_step on host numpy arrays (pinned memory moves fastest): the inputs
    go to the device, E comes back updated in place."""
    info = fld_info()
    st = lib().fld_step_host(ctx.handle, _hptr(E, ctx.n, "E"), _hptr(nHI, ctx.n, "n_HI"),
                             _hptr(eta, ctx.n, "eta"), ctypes.byref(info))
    if check:
        _check(st, "fld_step_host")
    d = info.as_dict()
    d["status"] = st
    return d


def fld_step_batched(ctxs: Sequence[Context], Es, nHIs, etas, check: bool = True):
    """Step independent contexts together (lockstep rounds, one graph launch
    per round); returns (status, [info dict per context])."""
    n = len(ctxs)
    arr = lambda xs: (_VP * n)(*xs)
    infos = (fld_info * n)()
    st = lib().fld_step_batched(n, arr([c.handle for c in ctxs]),
                                arr([_dptr(e, c.n, "E") for e, c in zip(Es, ctxs)]),
                                arr([_dptr(e, c.n, "n_HI") for e, c in zip(nHIs, ctxs)]),
                                arr([_dptr(e, c.n, "eta") for e, c in zip(etas, ctxs)]), infos)
    if check:
        _check(st, "fld_step_batched")
    return st, [i.as_dict() for i in infos]


def fld_apply(ctx: Context, x, y):
    """y = A x with the assembled FP64 operator (device tensors)."""
    _check(lib().fld_apply(ctx.handle, _dptr(x, ctx.n, "x"), _dptr(y, ctx.n, "y")), "fld_apply")


def fld_vcycle(ctx: Context, r, z):
    """z = one V-cycle applied to r (the preconditioner; FP32 on a mixed
    context, with r and z FP64 device tensors)."""
    _check(lib().fld_vcycle(ctx.handle, _dptr(r, ctx.n, "r"), _dptr(z, ctx.n, "z")), "fld_vcycle")


def fld_get_system(ctx: Context, m=None, wx=None, wy=None, wz=None, b=None):
    """Copy the assembled FP64 operator (m, wx, wy, wz) and right-hand side b
    into the given device tensors (None: skipped)."""
    ptrs = [None if t is None else _dptr(t, ctx.n) for t in (m, wx, wy, wz, b)]
    _check(lib().fld_get_system(ctx.handle, *ptrs), "fld_get_system")


def fld_opacity_update(E, nH, nHI, out, dt, c, sigma, hnu, alpha_B, stream=None):
    """n_HI after the hydrogen-only linearly implicit update of one step (the
    opacity update between radiation steps), into out."""
    import torch
    n = E.numel()
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().fld_opacity_update(n, _dptr(E, n, "E"), _dptr(nH, n, "n_H"), _dptr(nHI, n, "n_HI"),
                                    _dptr(out, n, "out"), float(dt), float(c), float(sigma),
                                    float(hnu), float(alpha_B), _VP(stream.cuda_stream)),
           "fld_opacity_update")


def fld_params_default() -> fld_params:
    """The library's default parameters."""
    p = fld_params()
    _check(lib().fld_params_default(ctypes.byref(p)), "fld_params_default")
    return p


def fld_profile(ctx: Context, class_mask: int = 0):
    """Reset launch statistics; time the kernel classes in class_mask."""
    _check(lib().fld_profile(ctx.handle, ctypes.c_ulonglong(class_mask)), "fld_profile")


def fld_profile_read(ctx: Context) -> List[dict]:
    """Per kernel class: launches, timed launches, ms and algorithmic bytes
    since the last fld_profile."""
    n = lib().fld_profile_read(ctx.handle, None, 0)
    arr = (fld_kernel_stat * n)()
    lib().fld_profile_read(ctx.handle, arr, n)
    out = []
    for i, k in enumerate(arr):
        out.append({"cls": i, "name": k.name.decode(), "launches": k.launches, "timed": k.timed,
                    "ms": k.ms, "bytes": k.bytes, "timed_bytes": k.timed_bytes})
    return out


def fld_set_dt(ctx: Context, dt: float):
    """Change the time step of the following steps."""
    _check(lib().fld_set_dt(ctx.handle, float(dt)), "fld_set_dt")


def fld_set_expansion(ctx: Context, scale_factor: float, adot_over_a: float):
    """Set the scale factor and the expansion rate adot/a (s^-1) of the
    following steps (comoving cell widths, cosmological loss term)."""
    _check(lib().fld_set_expansion(ctx.handle, float(scale_factor), float(adot_over_a)),
           "fld_set_expansion")


def fld_advance(ctx: Context, E, nHI, eta, t_span: float, dt_first: float, tau_tol: float = 1e-4,
                dt_min: float = 1e-6 * 3.15576e7, dt_max: float = 0.0, growth: float = 2.0,
                max_substeps: int = 10000, check: bool = True) -> dict:
    """Subcycled advance of E over t_span (see fld_advance in fld.h)."""
    ap = fld_advance_params(float(tau_tol), float(dt_min), float(dt_max), float(growth), int(max_substeps))
    info = fld_advance_info()
    st = lib().fld_advance(ctx.handle, _dptr(E, ctx.n, "E"), _dptr(nHI, ctx.n, "n_HI"), _dptr(eta, ctx.n, "eta"),
                           float(t_span), float(dt_first), ctypes.byref(ap), ctypes.byref(info))
    if check:
        _check(st, "fld_advance")
    d = info.as_dict()
    d["status"] = st
    return d


def fld_residual_noalloc(grid, m, wx, wy, wz, b, x, r, norms, stream=None):
    """r = b - A x and norms = [||r||^2, max |r|] with no device allocation
    (see fld_residual_noalloc in fld.h); r may be None."""
    import torch
    g = make_grid(grid)
    n = g.nx * g.ny * g.nz
    if stream is None:
        stream = torch.cuda.current_stream()
    ptrs = [_dptr(t, n, nm) for t, nm in ((m, "m"), (wx, "wx"), (wy, "wy"), (wz, "wz"), (b, "b"), (x, "x"))]
    rp = None if r is None else _dptr(r, n, "r")
    _check(lib().fld_residual_noalloc(ctypes.byref(g), *ptrs, rp, _dptr(norms, 2, "norms"),
                                      _VP(stream.cuda_stream)), "fld_residual_noalloc")


def fld_autotune(ctx: Context, reps: int = 3):
    """Time the candidate launch shapes and prefetch distances of the FP32
    sweeps on this context and keep the fastest (mixed contexts only)."""
    _check(lib().fld_autotune(ctx.handle, int(reps)), "fld_autotune")


def fld_tuning_size(ctx: Context) -> int:
    """Length of the tuning table (three ints per kernel and level)."""
    return int(lib().fld_tuning_size(ctx.handle))


def fld_get_tuning(ctx: Context) -> List[int]:
    """The tuning table: (threads, target blocks, prefetch distance) per
    kernel and level."""
    n = fld_tuning_size(ctx)
    buf = (ctypes.c_int * n)()
    _check(lib().fld_get_tuning(ctx.handle, buf, n), "fld_get_tuning")
    return list(buf)


def fld_set_tuning(ctx: Context, table: Sequence[int]):
    """Install a tuning table (e.g. from another context of the same grid)."""
    buf = (ctypes.c_int * len(table))(*[int(v) for v in table])
    _check(lib().fld_set_tuning(ctx.handle, buf, len(table)), "fld_set_tuning")


def autotune(ctx: Context, cache_path: Optional[str] = None, reps: int = 3) -> List[int]:
    """Tune the context's FP32 launch shapes, or load them from a JSON cache
    keyed by grid, boundaries, precision and GPU name; returns the table."""
    import json
    import torch
    g = ctx._g
    key = "%dx%dx%d_bc%d%d%d_p%d_%s" % (g.nx, g.ny, g.nz, g.bc[0], g.bc[1], g.bc[2], ctx.params.precision,
                                         torch.cuda.get_device_name().replace(" ", "_"))
    if cache_path is None:
        cache_path = os.environ.get("FLD_TUNE_CACHE",
                                    os.path.join(os.path.expanduser("~"), ".cache", "fld_gb300_tuning.json"))
    cache = {}
    try:
        with open(cache_path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    table = cache.get(key)
    if table is not None and len(table) == fld_tuning_size(ctx):
        fld_set_tuning(ctx, table)
        return table
    fld_autotune(ctx, reps)
    table = fld_get_tuning(ctx)
    cache[key] = table
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f)
    except OSError:
        pass
    return table


# ------------------------------------------------------------ spectral model

def fld_sed_default(**overrides) -> fld_sed:
    """SED record: the library's defaults with fields overridden by keyword
    (kind, nu_mono, T, alpha)."""
    sed = fld_sed()
    _check(lib().fld_sed_default(ctypes.byref(sed)), "fld_sed_default")
    for k, v in overrides.items():
        setattr(sed, k, type(getattr(sed, k))(v))
    return sed


def fld_sed_integrals(sed: fld_sed, edges: Sequence[float], stream=None) -> np.ndarray:
    """Coefficient table (groups x FLD_SED_NCOEF) for frequency-group edges (Hz)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    groups = e.size - 1
    coef = np.zeros((max(groups, 1), FLD_SED_NCOEF))
    st = lib().fld_sed_integrals(ctypes.byref(sed), ctypes.c_void_p(e.ctypes.data), int(groups),
                                 ctypes.c_void_p(coef.ctypes.data), _stream(stream))
    _check(st, "fld_sed_integrals")
    return coef


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _VP(s.cuda_stream)


def _ptrs(ts, n, what):
    arr = (_VP * len(ts))()
    for g, t in enumerate(ts):
        arr[g] = _dptr(t, n, f"{what}[{g}]").value
    return arr


def _opt(t, n, what):
    return _dptr(t, n, what) if t is not None else None


def fld_group_fields(coef: np.ndarray, n_HI, kappas, n_HeI=None, n_HeII=None, eta=None, etas=None,
                     stream=None):
    """kappa_g = sum_i n_i K_gi and eta_g = F_g eta into the given tensors."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    groups = coef.shape[0]
    n = n_HI.numel()
    st = lib().fld_group_fields(n, groups, ctypes.c_void_p(coef.ctypes.data), _dptr(n_HI, n, "n_HI"),
                                _opt(n_HeI, n, "n_HeI"), _opt(n_HeII, n, "n_HeII"), _opt(eta, n, "eta"),
                                ctypes.cast(_ptrs(kappas, n, "kappa"), _VP),
                                ctypes.cast(_ptrs(etas, n, "eta_out"), _VP) if etas is not None else None,
                                _stream(stream))
    _check(st, "fld_group_fields")


def fld_photo_rates(coef: np.ndarray, E_groups, n_HI=None, n_HeI=None, n_HeII=None, rho_b=None,
                    c_light=2.99792458e10, gamma_HI=None, gamma_HeI=None, gamma_HeII=None, heating=None,
                    stream=None):
    """Photoionisation rates of HI, HeI, HeII and the photoheating rate from the
    group energies E_groups and the group integrals coef (fld_sed_integrals),
    into the given device tensors (None: not computed)."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    groups = coef.shape[0]
    n = E_groups[0].numel()
    st = lib().fld_photo_rates(n, groups, ctypes.c_void_p(coef.ctypes.data),
                               ctypes.cast(_ptrs(E_groups, n, "E"), _VP), _opt(n_HI, n, "n_HI"),
                               _opt(n_HeI, n, "n_HeI"), _opt(n_HeII, n, "n_HeII"), _opt(rho_b, n, "rho_b"),
                               float(c_light), _opt(gamma_HI, n, "gamma_HI"), _opt(gamma_HeI, n, "gamma_HeI"),
                               _opt(gamma_HeII, n, "gamma_HeII"), _opt(heating, n, "heating"), _stream(stream))
    _check(st, "fld_photo_rates")
