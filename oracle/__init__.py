"""FP64 CPU oracle for the implicit grey FLD radiation step (ctypes binding).

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg are the only users.  The product library never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``fld_oracle.c`` (plain C, FP64, one OpenMP loop per
stencil sweep, serial dot products); see that file's header for the paper
passages it follows (Sec. 2 limiter, Sec. 3.2 theta-method correction
system, Table 1 solver) and the readings taken where the paper is silent.

Arrays are numpy float64, C-contiguous, shaped (nz, ny, nx) so that x is the
fastest index.  Parameters are passed as any object (or dict) with the
attribute names used below.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fld_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOCONV = 0, 1, 2, 3
LIMITER_PAPER, LIMITER_LP = 0, 1
SMOOTH_RBGS, SMOOTH_JACOBI = 0, 1


class OracleError(RuntimeError):
    """A failed oracle call (its C status code and the call's name)."""

    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (IEEE arithmetic, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("dirichlet", ctypes.c_int * 6),
                ("ebc", ctypes.c_double * 6)]


class _Phys(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("c", ctypes.c_double),
                ("L_unit", ctypes.c_double), ("dmax_coef", ctypes.c_double),
                ("rmin_coef", ctypes.c_double), ("sigma", ctypes.c_double),
                ("adot", ctypes.c_double), ("hnu", ctypes.c_double),
                ("limiter", ctypes.c_int), ("theta", ctypes.c_double), ("a", ctypes.c_double)]


class _Solver(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("omega", ctypes.c_double),
                ("pre", ctypes.c_int), ("post", ctypes.c_int),
                ("rtol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("coarse_cap", ctypes.c_int), ("paper_order", ctypes.c_int)]


_P = ctypes.POINTER(ctypes.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            for name, args, res in [
                ("or_num_threads", [], ctypes.c_int),
                ("or_lp_lambda", [ctypes.c_double], ctypes.c_double),
                ("or_face_D", [ctypes.c_double] * 5 + [ctypes.POINTER(_Phys)], ctypes.c_double),
                ("or_assemble", [ctypes.POINTER(_Grid), ctypes.POINTER(_Phys)] + [_P] * 9, ctypes.c_int),
                ("or_bnd_size", [ctypes.POINTER(ctypes.c_int)], ctypes.c_size_t),
                ("or_apply", [ctypes.POINTER(_Grid)] + [_P] * 6, None),
                ("or_dense_matrix", [ctypes.POINTER(_Grid)] + [_P] * 5, ctypes.c_int),
                ("or_dense_solve", [ctypes.POINTER(_Grid)] + [_P] * 6, ctypes.c_int),
                ("or_vcycle", [ctypes.POINTER(_Grid)] + [_P] * 7 + [ctypes.POINTER(_Solver)], ctypes.c_int),
                ("or_pcg", [ctypes.POINTER(_Grid)] + [_P] * 7 + [ctypes.POINTER(_Solver),
                            ctypes.POINTER(ctypes.c_int), _P, _P], ctypes.c_int),
                ("or_step", [ctypes.POINTER(_Grid), ctypes.POINTER(_Phys), ctypes.POINTER(_Solver)]
                 + [_P] * 5, ctypes.c_int),
                ("or_num_levels", [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
                ("or_coarsen", [ctypes.POINTER(ctypes.c_int)] * 3 + [_P] * 10, ctypes.c_int),
                ("or_prolong_add", [ctypes.POINTER(ctypes.c_int)] * 2 + [_P] * 2, ctypes.c_int),
                ("or_restrict", [ctypes.POINTER(ctypes.c_int)] * 2 + [_P] * 2, ctypes.c_int),
                ("or_opacity_update", [ctypes.c_size_t] + [_P] * 4 + [ctypes.c_double] * 5, ctypes.c_int),
                ("or_advance", [ctypes.POINTER(_Grid), ctypes.POINTER(_Phys), ctypes.POINTER(_Solver)]
                 + [_P] * 3 + [ctypes.c_double] * 6 + [ctypes.c_int, _P], ctypes.c_int),
            ]:
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _get(obj, name, default=None):
    if isinstance(obj, dict):
        return obj.get(name, default)
    return getattr(obj, name, default)


def _dirichlet(g):
    """Per-side Dirichlet flags and values (x lo, x hi, y lo, y hi, z lo, z hi)
    of a grid object: attributes ``dirichlet`` (6 flags) and ``ebc`` (6
    values); absent means reflecting everywhere."""
    d = _get(g, "dirichlet") or (0,) * 6
    v = _get(g, "ebc") or (0.0,) * 6
    return [1 if x else 0 for x in d], [float(x) for x in v]


def _has_dirichlet(g) -> bool:
    return any(_dirichlet(g)[0])


def _grid(g) -> _Grid:
    n = _get(g, "n")
    h = _get(g, "h")
    per = _get(g, "periodic")
    dflag, dval = _dirichlet(g)
    return _Grid((ctypes.c_int * 3)(*[int(v) for v in n]),
                 (ctypes.c_double * 3)(*[float(v) for v in h]),
                 (ctypes.c_int * 3)(*[1 if v else 0 for v in per]),
                 (ctypes.c_int * 6)(*dflag), (ctypes.c_double * 6)(*dval))


def _phys(p) -> _Phys:
    return _Phys(float(_get(p, "dt")), float(_get(p, "c")), float(_get(p, "L_unit")),
                 float(_get(p, "dmax_coef", 0.006)), float(_get(p, "rmin_coef", 1e-20)),
                 float(_get(p, "sigma")), float(_get(p, "adot_over_a", 0.0)),
                 float(_get(p, "hnu", 2.17896e-11)), int(_get(p, "limiter", LIMITER_PAPER)),
                 float(_get(p, "theta", 1.0)), float(_get(p, "scale_factor", 1.0)))


def _solver(s) -> _Solver:
    return _Solver(int(_get(s, "smoother", SMOOTH_RBGS)), float(_get(s, "jacobi_omega", 0.8)),
                   int(_get(s, "pre", 1)), int(_get(s, "post", 1)),
                   float(_get(s, "rtol", 1e-8)), int(_get(s, "max_iter", 50)),
                   int(_get(s, "coarse_cap", 1024)), int(_get(s, "paper_order", 0)))


def _arr(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _optr(a):
    return _ptr(a) if a is not None else None


def bnd_size(n) -> int:
    """Length of the packed Dirichlet face array of an n = (nx, ny, nz) grid."""
    return int(_lib_handle().or_bnd_size((ctypes.c_int * 3)(*[int(v) for v in n])))


def _shape(g):
    n = _get(g, "n")
    return (int(n[2]), int(n[1]), int(n[0]))


def num_threads() -> int:
    """OpenMP threads the oracle runs with."""
    return _lib_handle().or_num_threads()


def lp_lambda(x: float) -> float:
    """Levermore-Pomraning lambda(x) = (coth x - 1/x) / x (series for small x)."""
    return _lib_handle().or_lp_lambda(float(x))


def face_D(E1, E2, k1, k2, h, phys) -> float:
    """Limited diffusion coefficient of one face between cells with energies
    E1, E2 and opacities k1, k2, spacing h (Sec. 2)."""
    p = _phys(phys)
    return _lib_handle().or_face_D(float(E1), float(E2), float(k1), float(k2), float(h),
                                   ctypes.byref(p))


def assemble(grid, phys, E, nHI, eta) -> dict:
    """Operator (m, wx, wy, wz), the packed Dirichlet face weights "bnd" (None
    when the grid has no Dirichlet side) and the right-hand side b of
    A dE = b."""
    sh = _shape(grid)
    E, nHI, eta = _arr(E, sh), _arr(nHI, sh), _arr(eta, sh)
    out = {k: np.empty(sh) for k in ("m", "wx", "wy", "wz", "b")}
    out["bnd"] = np.empty(bnd_size(_get(grid, "n"))) if _has_dirichlet(grid) else None
    g, p = _grid(grid), _phys(phys)
    st = _lib_handle().or_assemble(ctypes.byref(g), ctypes.byref(p), _ptr(E), _ptr(nHI), _ptr(eta),
                                   _ptr(out["m"]), _ptr(out["wx"]), _ptr(out["wy"]),
                                   _ptr(out["wz"]), _ptr(out["b"]), _optr(out["bnd"]))
    if st:
        raise OracleError(st, "assemble")
    return out


def _op(grid, op):
    sh = _shape(grid)
    return [_arr(op[k], sh) for k in ("m", "wx", "wy", "wz")]


def _bnd(grid, op):
    b = op.get("bnd") if isinstance(op, dict) else None
    if b is None:
        return None
    return _arr(b).ravel()


def apply(grid, op, x) -> np.ndarray:
    """A x for the assembled operator op (m, wx, wy, wz)."""
    sh = _shape(grid)
    m, wx, wy, wz = _op(grid, op)
    x = _arr(x, sh)
    y = np.empty(sh)
    g = _grid(grid)
    _lib_handle().or_apply(ctypes.byref(g), _ptr(m), _ptr(wx), _ptr(wy), _ptr(wz), _ptr(x), _ptr(y))
    return y


def dense_matrix(grid, op) -> np.ndarray:
    """The operator as a dense n x n matrix (small grids)."""
    m, wx, wy, wz = _op(grid, op)
    n = m.size
    A = np.empty((n, n))
    g = _grid(grid)
    _lib_handle().or_dense_matrix(ctypes.byref(g), _ptr(m), _ptr(wx), _ptr(wy), _ptr(wz), _ptr(A))
    return A


def dense_solve(grid, op, rhs) -> np.ndarray:
    """A^-1 rhs by dense Cholesky (small grids)."""
    sh = _shape(grid)
    m, wx, wy, wz = _op(grid, op)
    rhs = _arr(rhs, sh)
    x = np.empty(sh)
    g = _grid(grid)
    st = _lib_handle().or_dense_solve(ctypes.byref(g), _ptr(m), _ptr(wx), _ptr(wy), _ptr(wz),
                                      _ptr(rhs), _ptr(x))
    if st:
        raise OracleError(st, "dense_solve")
    return x


def vcycle(grid, op, r, solver=None) -> np.ndarray:
    """One V-cycle of the multigrid preconditioner applied to r (solver: the
    smoother, pre/post sweeps and coarsest-grid options)."""
    sh = _shape(grid)
    m, wx, wy, wz = _op(grid, op)
    r = _arr(r, sh)
    z = np.empty(sh)
    g, s = _grid(grid), _solver(solver or {})
    bnd = _bnd(grid, op)
    st = _lib_handle().or_vcycle(ctypes.byref(g), _ptr(m), _ptr(wx), _ptr(wy), _ptr(wz),
                                 _optr(bnd), _ptr(r), _ptr(z), ctypes.byref(s))
    if st:
        raise OracleError(st, "vcycle")
    return z


def pcg(grid, op, b, solver=None, allow_noconv=False):
    """MG-PCG solve; returns (x, iters, true relative residual, history)."""
    sh = _shape(grid)
    m, wx, wy, wz = _op(grid, op)
    b = _arr(b, sh)
    x = np.empty(sh)
    s = _solver(solver or {})
    g = _grid(grid)
    iters = ctypes.c_int(0)
    rel = np.zeros(1)
    hist = np.zeros(s.max_iter + 1)
    bnd = _bnd(grid, op)
    st = _lib_handle().or_pcg(ctypes.byref(g), _ptr(m), _ptr(wx), _ptr(wy), _ptr(wz), _optr(bnd),
                              _ptr(b), _ptr(x), ctypes.byref(s), ctypes.byref(iters), _ptr(rel),
                              _ptr(hist))
    if st and not (st == ENOCONV and allow_noconv):
        raise OracleError(st, "pcg")
    return x, iters.value, float(rel[0]), hist[: iters.value + 1]


def step(grid, phys, solver, E, nHI, eta, allow_noconv=False):
    """One FLD theta-method step: returns (E_new, info dict)."""
    sh = _shape(grid)
    E, nHI, eta = _arr(E, sh), _arr(nHI, sh), _arr(eta, sh)
    E_new = E.copy()
    info = np.zeros(9)
    g, p, s = _grid(grid), _phys(phys), _solver(solver or {})
    st = _lib_handle().or_step(ctypes.byref(g), ctypes.byref(p), ctypes.byref(s), _ptr(E),
                               _ptr(nHI), _ptr(eta), _ptr(E_new), _ptr(info))
    if st and not (st == ENOCONV and allow_noconv):
        raise OracleError(st, "step")
    return E_new, {"status": st, "iters": int(info[0]), "rel_res": info[1],
                   "balance_abs": info[2], "balance_rel": info[3],
                   "emitted": info[4], "absorbed": info[5], "floor_added": info[6],
                   "rel_change": info[7], "outflow": info[8]}


def num_levels(n):
    """The multigrid level shapes of an nx x ny x nz grid, finest first."""
    dims = (ctypes.c_int * 96)()
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    nl = _lib_handle().or_num_levels(nn, dims)
    return [tuple(dims[3 * l: 3 * l + 3]) for l in range(nl)]


def _ints(v):
    return (ctypes.c_int * 3)(*[int(x) for x in v])


def coarsen(nf, periodic, op, dirichlet=None):
    """Coarse operator of a level; with dirichlet (6 flags) the op's packed
    face weights "bnd" are coarsened too."""
    shf = (nf[2], nf[1], nf[0])
    shc = (nf[2] // 2, nf[1] // 2, nf[0] // 2)
    ins = [_arr(op[k], shf) for k in ("m", "wx", "wy", "wz")]
    outs = {k: np.empty(shc) for k in ("m", "wx", "wy", "wz")}
    dflag = None
    bnd = bndc = None
    if dirichlet is not None and any(dirichlet):
        dflag = (ctypes.c_int * 6)(*[1 if v else 0 for v in dirichlet])
        bnd = _arr(op["bnd"]).ravel()
        bndc = np.empty(bnd_size((nf[0] // 2, nf[1] // 2, nf[2] // 2)))
    st = _lib_handle().or_coarsen(_ints(nf), _ints(periodic), dflag, *[_ptr(a) for a in ins], _optr(bnd),
                                  *[_ptr(outs[k]) for k in ("m", "wx", "wy", "wz")], _optr(bndc))
    if st:
        raise OracleError(st, "coarsen")
    outs["bnd"] = bndc
    return outs


def prolong_add(nf, periodic, ec, zf):
    """zf + P ec: trilinear prolongation of the coarse array ec onto the fine
    array zf (fine shape nf)."""
    shf = (nf[2], nf[1], nf[0])
    shc = (nf[2] // 2, nf[1] // 2, nf[0] // 2)
    ec = _arr(ec, shc)
    z = _arr(zf, shf).copy()
    _lib_handle().or_prolong_add(_ints(nf), _ints(periodic), _ptr(ec), _ptr(z))
    return z


def restrict(nf, periodic, rf):
    """R rf = P^T rf / 8: full-weighting restriction of the fine array rf."""
    shf = (nf[2], nf[1], nf[0])
    shc = (nf[2] // 2, nf[1] // 2, nf[0] // 2)
    rf = _arr(rf, shf)
    rc = np.empty(shc)
    _lib_handle().or_restrict(_ints(nf), _ints(periodic), _ptr(rf), _ptr(rc))
    return rc


def opacity_update(E, nH, nHI, dt, c, sigma, hnu, alpha_B):
    """n_HI after one hydrogen-only linearly implicit backward-Euler update of the
    ionised fraction (one Jacobi iteration, clamped to [1e-12, 1])."""
    E, nH, nHI = _arr(E), _arr(nH), _arr(nHI)
    out = np.empty_like(nHI)
    _lib_handle().or_opacity_update(nHI.size, _ptr(E), _ptr(nH), _ptr(nHI), _ptr(out),
                                    float(dt), float(c), float(sigma), float(hnu), float(alpha_B))
    return out


def advance(grid, phys, solver, E, nHI, eta, t_span, dt_first, tau_tol=1e-4, dt_min=3.15576e1,
            dt_max=0.0, growth=2.0, max_substeps=10000, allow_fail=False):
    """Subcycled advance over t_span; returns (E, info dict)."""
    sh = _shape(grid)
    E = _arr(E, sh).copy()
    nHI, eta = _arr(nHI, sh), _arr(eta, sh)
    out = np.zeros(5)
    g, p, s = _grid(grid), _phys(phys), _solver(solver or {})
    st = _lib_handle().or_advance(ctypes.byref(g), ctypes.byref(p), ctypes.byref(s), _ptr(E), _ptr(nHI),
                                  _ptr(eta), float(t_span), float(dt_first), float(tau_tol), float(dt_min),
                                  float(dt_max), float(growth), int(max_substeps), _ptr(out))
    if st and not allow_fail:
        raise OracleError(st, "advance")
    return E, {"status": st, "substeps": int(out[0]), "retries": int(out[1]), "iters": int(out[2]),
               "t_done": out[3], "dt_next": out[4]}
