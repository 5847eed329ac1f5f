"""Python binding of the C ABI in include/qdd.h (argument marshalling only).

Every function here forwards to the entry point of the same name in
libqdd.so; all arithmetic runs in that library's CUDA kernels.  Arrays may be
torch tensors (CUDA or CPU, pinned or not) or numpy arrays, complex128 in the
canonical layouts:

    spinor  [V][4][3]       (V = Lx Ly Lz Lt, site x + Lx (y + Ly (z + Lz t)))
    gauge   [V][4][3][3]

There is no fallback: if the library is missing or fails to load, importing
this module raises, so a missing build can never be mistaken for a result.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqdd.so")

QDD_OK = 0
QDD_ERR_ARG = 1
QDD_ERR_CUDA = 2
QDD_ERR_NOMEM = 3
QDD_ERR_NOT_CONVERGED = 4
QDD_ERR_BREAKDOWN = 5
QDD_ERR_NONFINITE = 6
QDD_ERR_TIMEOUT = 7
QDD_ERR_STATE = 8
STATUS_NAMES = {0: "QDD_OK", 1: "QDD_ERR_ARG", 2: "QDD_ERR_CUDA", 3: "QDD_ERR_NOMEM", 4: "QDD_ERR_NOT_CONVERGED",
                5: "QDD_ERR_BREAKDOWN", 6: "QDD_ERR_NONFINITE", 7: "QDD_ERR_TIMEOUT", 8: "QDD_ERR_STATE"}

QDD_F64, QDD_F32, QDD_F16 = 0, 1, 2
PREC = {"f64": QDD_F64, "f32": QDD_F32, "f16": QDD_F16, QDD_F64: QDD_F64, QDD_F32: QDD_F32, QDD_F16: QDD_F16}
# qdd_schwarz: the member of the Schwarz family used as the preconditioner
QDD_SCHWARZ_RAS, QDD_SCHWARZ_SAP, QDD_SCHWARZ_AS = 0, 1, 2
SCHWARZ = {"ras": QDD_SCHWARZ_RAS, "sap": QDD_SCHWARZ_SAP, "as": QDD_SCHWARZ_AS}

# Every function the header declares (checked by the tests against the library's exports).
ABI = ("qdd_version", "qdd_last_error", "qdd_default_params", "qdd_create_lattice", "qdd_destroy_lattice",
       "qdd_load_gauge", "qdd_dslash", "qdd_ras_apply", "qdd_solve", "qdd_field_create", "qdd_field_destroy",
       "qdd_field_import", "qdd_field_export", "qdd_dslash_field", "qdd_kernel_launches", "qdd_set_profiling",
       "qdd_profile_read", "qdd_measure_fma_peak", "qdd_ras_field_noalloc", "qdd_autotune", "qdd_solve_batch",
       "qdd_solve_batch_each", "qdd_tuned_params", "qdd_load_gauge_clover", "qdd_set_batch_lists",
       "qdd_test_ras_wait")

# Kernel classes of the per-class GPU timers (qdd_profile).
KCLASS = ("dslash", "dslash_f64", "ras", "blas", "convert", "clover")


class QddError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SolverParams(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int * 4), ("overlap", ctypes.c_int), ("n_dominv", ctypes.c_int),
                ("n_ras", ctypes.c_int), ("inner_prec", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_inner", ctypes.c_int), ("max_outer", ctypes.c_int), ("use_ras", ctypes.c_int),
                ("outer_mode", ctypes.c_int), ("autotune", ctypes.c_int), ("ras_kernel", ctypes.c_int),
                ("schwarz", ctypes.c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 6), ("launches", ctypes.c_longlong * 6)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("dv_count", ctypes.c_int),
                ("ras_sweeps", ctypes.c_int), ("status", ctypes.c_int), ("true_rel_residual", ctypes.c_double),
                ("t_total_ms", ctypes.c_double), ("t_outer_ms", ctypes.c_double), ("t_inner_ms", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1011_3318_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I4 = ctypes.POINTER(ctypes.c_int)
    st = ctypes.c_int
    lib.qdd_version.restype = ctypes.c_char_p
    lib.qdd_last_error.restype = ctypes.c_char_p
    lib.qdd_default_params.argtypes = [ctypes.POINTER(SolverParams)]
    lib.qdd_default_params.restype = None
    lib.qdd_create_lattice.argtypes = [ctypes.POINTER(P), I4, I4, ctypes.c_int, P]
    lib.qdd_destroy_lattice.argtypes = [P]
    lib.qdd_load_gauge.argtypes = [P, P]
    lib.qdd_load_gauge_clover.argtypes = [P, P, ctypes.c_double, ctypes.c_double]
    lib.qdd_dslash.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.qdd_ras_apply.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(SolverParams)]
    lib.qdd_solve.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo)]
    lib.qdd_field_create.argtypes = [P, ctypes.c_int, ctypes.POINTER(P)]
    lib.qdd_field_destroy.argtypes = [P]
    lib.qdd_field_import.argtypes = [P, P]
    lib.qdd_field_export.argtypes = [P, P]
    lib.qdd_dslash_field.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double]
    lib.qdd_kernel_launches.restype = ctypes.c_ulonglong
    lib.qdd_set_profiling.argtypes = [P, ctypes.c_int]
    lib.qdd_profile_read.argtypes = [P, ctypes.POINTER(Profile), ctypes.c_int]
    lib.qdd_measure_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.qdd_test_ras_wait.argtypes = [ctypes.c_uint, ctypes.c_long]
    lib.qdd_solve_batch.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                    ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo)]
    lib.qdd_solve_batch_each.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_double, ctypes.POINTER(ctypes.POINTER(SolverParams)),
                                         ctypes.POINTER(SolveInfo)]
    lib.qdd_tuned_params.argtypes = [P, ctypes.POINTER(SolverParams)]
    lib.qdd_set_batch_lists.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.qdd_autotune.argtypes = [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(SolverParams), ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.qdd_ras_field_noalloc.argtypes = [P, P, P, P, P, ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(SolverParams)]
    for name in ABI:
        if name not in ("qdd_version", "qdd_last_error", "qdd_default_params", "qdd_kernel_launches"):
            getattr(lib, name).restype = st
    return lib


_lib = _load()


def lib():
    return _lib


def version() -> str:
    return _lib.qdd_version().decode()


def last_error() -> str:
    return _lib.qdd_last_error().decode()


def _check(status: int, what: str, allow=()):
    if status != QDD_OK and status not in allow:
        raise QddError(status, what, last_error())
    return status


def _ptr(a, writable: bool = False):
    """(pointer, keepalive) of a complex128 array or tensor, contiguous."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.complex128 or not a.is_contiguous():
                raise TypeError("tensors must be contiguous complex128")
            return a.data_ptr(), a
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if a.dtype != np.complex128 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be C-contiguous complex128")
        if writable and not a.flags["WRITEABLE"]:
            raise TypeError("output array is read-only")
        return a.ctypes.data, a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Lattice:
    """Handle of a qdd_lattice (create with create_lattice)."""

    def __init__(self, handle, dims, bc, n_rhs=1, stream=None):
        self.handle = handle
        self.dims = tuple(dims)
        self.bc = tuple(bc)
        self.V = int(np.prod(dims))
        self.n_rhs = int(n_rhs)
        self.stream = stream  # kept alive with the lattice

    def __del__(self):
        try:
            destroy_lattice(self)
        except Exception:
            pass


def default_params(**overrides) -> SolverParams:
    p = SolverParams()
    _lib.qdd_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "block":
            p.block = (ctypes.c_int * 4)(*[int(b) for b in v])
        elif k == "inner_prec":
            p.inner_prec = PREC[v]
        elif k == "schwarz" and isinstance(v, str):
            p.schwarz = SCHWARZ[v]
        else:
            setattr(p, k, v)
    return p


def create_lattice(dims, bc=(1, 1, 1, -1), n_rhs: int = 1, stream=None) -> Lattice:
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    b = (ctypes.c_int * 4)(*[int(x) for x in bc])
    _check(_lib.qdd_create_lattice(ctypes.byref(h), d, b, int(n_rhs), _stream_handle(stream)), "qdd_create_lattice")
    return Lattice(h, dims, bc, n_rhs, stream)


def destroy_lattice(lat: Lattice) -> None:
    if lat.handle:
        _lib.qdd_destroy_lattice(lat.handle)
        lat.handle = None


def load_gauge(lat: Lattice, U, kappa: float | None = None, c_sw: float | None = None) -> None:
    """Load the links; with kappa and c_sw also build the clover term in the
    same pass (qdd_load_gauge_clover)."""
    p, _keep = _ptr(U)
    if kappa is None and c_sw is None:
        _check(_lib.qdd_load_gauge(lat.handle, p), "qdd_load_gauge")
    else:
        _check(_lib.qdd_load_gauge_clover(lat.handle, p, float(kappa), float(c_sw)), "qdd_load_gauge_clover")


def dslash(lat: Lattice, out, inp, kappa: float, c_sw: float, prec="f64") -> None:
    po, _k1 = _ptr(out, True)
    pi, _k2 = _ptr(inp)
    _check(_lib.qdd_dslash(lat.handle, po, pi, float(kappa), float(c_sw), PREC[prec]), "qdd_dslash")


def ras_apply(lat: Lattice, out, inp, kappa: float, c_sw: float, params: SolverParams) -> None:
    po, _k1 = _ptr(out, True)
    pi, _k2 = _ptr(inp)
    _check(_lib.qdd_ras_apply(lat.handle, po, pi, float(kappa), float(c_sw), ctypes.byref(params)), "qdd_ras_apply")


def _info_dicts(infos, st):
    out = []
    for info in infos:
        d = {k: getattr(info, k) for k, _ in SolveInfo._fields_}
        d["return_status"] = st
        out.append(d)
    return out


def solve(lat: Lattice, phi, eta, kappa: float, c_sw: float, tol: float, params: SolverParams | None = None,
          raise_on_failure: bool = True):
    """Solve D phi = eta; returns the info dict (a list of them, one per
    right-hand side, when the lattice has n_rhs > 1)."""
    po, _k1 = _ptr(phi, True)
    pe, _k2 = _ptr(eta)
    infos = (SolveInfo * lat.n_rhs)()
    st = _lib.qdd_solve(lat.handle, po, pe, float(kappa), float(c_sw), float(tol),
                        ctypes.byref(params) if params is not None else None, infos)
    if raise_on_failure:
        _check(st, "qdd_solve")
    out = _info_dicts(infos, st)
    return out[0] if lat.n_rhs == 1 else out


def solve_batch(lats, phis, etas, kappas, c_sws, tol: float, params=None, raise_on_failure: bool = True):
    """Solve independent systems (one per lattice) in lockstep; returns one
    list of info dicts per lattice.  params: one SolverParams for every
    lattice (qdd_solve_batch), or a list with one SolverParams or None per
    lattice (qdd_solve_batch_each: None takes the tuning cache's parameters
    for that lattice's shape, else the defaults)."""
    n = len(lats)
    keep = []
    ph = (ctypes.c_void_p * n)()
    et = (ctypes.c_void_p * n)()
    hs = (ctypes.c_void_p * n)(*[l.handle.value if isinstance(l.handle, ctypes.c_void_p) else l.handle for l in lats])
    for i in range(n):
        ph[i], k1 = _ptr(phis[i], True)
        et[i], k2 = _ptr(etas[i])
        keep += [k1, k2]
    ka = (ctypes.c_double * n)(*[float(k) for k in kappas])
    cs = (ctypes.c_double * n)(*[float(c) for c in c_sws])
    total = sum(l.n_rhs for l in lats)
    infos = (SolveInfo * total)()
    if isinstance(params, (list, tuple)):
        if len(params) != n:
            raise ValueError("one parameter set (or None) per lattice")
        pp = (ctypes.POINTER(SolverParams) * n)(*[ctypes.pointer(p) if p is not None else None for p in params])
        st = _lib.qdd_solve_batch_each(hs, ph, et, n, ka, cs, float(tol), pp, infos)
        what = "qdd_solve_batch_each"
    else:
        st = _lib.qdd_solve_batch(hs, ph, et, n, ka, cs, float(tol),
                                  ctypes.byref(params) if params is not None else None, infos)
        what = "qdd_solve_batch"
    if raise_on_failure:
        _check(st, what)
    flat = _info_dicts(infos, st)
    out, o = [], 0
    for l in lats:
        out.append(flat[o:o + l.n_rhs])
        o += l.n_rhs
    return out


def autotune(lat: Lattice, eta, kappa: float, c_sw: float, tol: float, params: SolverParams | None = None,
             max_trials: int = 40):
    """Best RAS parameters for solving D phi = eta (timed whole solves);
    returns (params, best_ms)."""
    p = params if params is not None else default_params()
    pe, _k = _ptr(eta)
    best = ctypes.c_double()
    _check(_lib.qdd_autotune(lat.handle, pe, float(kappa), float(c_sw), float(tol), ctypes.byref(p), int(max_trials),
                             ctypes.byref(best)), "qdd_autotune")
    return p, best.value


def tuned_params(lat: Lattice):
    """The tuning cache's parameters for this lattice's shape (set by
    autotune on a lattice of the same extents, boundary signs and
    right-hand-side count), or None."""
    p = SolverParams()
    st = _lib.qdd_tuned_params(lat.handle, ctypes.byref(p))
    if st == QDD_ERR_STATE:
        return None
    _check(st, "qdd_tuned_params")
    return p


def set_batch_lists(on: bool) -> bool:
    """Turns the batch work lists (qdd_set_batch_lists) on or off; returns
    the previous setting."""
    prev = ctypes.c_int(0)
    _check(_lib.qdd_set_batch_lists(1 if on else 0, ctypes.byref(prev)), "qdd_set_batch_lists")
    return bool(prev.value)


class Field:
    """Handle of a qdd_field (internal GPU layout of one precision)."""

    def __init__(self, handle, lat, prec):
        self.handle = handle
        self.lat = lat
        self.prec = prec

    def __del__(self):
        try:
            field_destroy(self)
        except Exception:
            pass


def field_create(lat: Lattice, prec="f32") -> Field:
    h = ctypes.c_void_p()
    _check(_lib.qdd_field_create(lat.handle, PREC[prec], ctypes.byref(h)), "qdd_field_create")
    return Field(h, lat, PREC[prec])


def field_destroy(f: Field) -> None:
    if f.handle:
        _lib.qdd_field_destroy(f.handle)
        f.handle = None


def field_import(f: Field, src) -> None:
    p, _k = _ptr(src)
    _check(_lib.qdd_field_import(f.handle, p), "qdd_field_import")


def field_export(f: Field, dst) -> None:
    p, _k = _ptr(dst, True)
    _check(_lib.qdd_field_export(f.handle, p), "qdd_field_export")


def dslash_field(lat: Lattice, out: Field, inp: Field, kappa: float, c_sw: float) -> None:
    _check(_lib.qdd_dslash_field(lat.handle, out.handle, inp.handle, float(kappa), float(c_sw)), "qdd_dslash_field")


def kernel_launches() -> int:
    """Process-wide number of kernel launches made by the library."""
    return int(_lib.qdd_kernel_launches())


def set_profiling(lat: Lattice, on: bool) -> None:
    _check(_lib.qdd_set_profiling(lat.handle, int(bool(on))), "qdd_set_profiling")


def profile_read(lat: Lattice, reset: bool = True) -> dict:
    """{class: (ms, launches)} of GPU time per kernel class since the last reset."""
    p = Profile()
    _check(_lib.qdd_profile_read(lat.handle, ctypes.byref(p), int(bool(reset))), "qdd_profile_read")
    return {k: (p.ms[i], p.launches[i]) for i, k in enumerate(KCLASS)}


def test_ras_wait(extra_bytes: int = 0, max_polls: int = 0) -> None:
    """Test support: bound the TMA-staged RAS sweep's wait to max_polls polls
    and make it expect extra_bytes that never arrive (0, 0: defaults)."""
    _check(_lib.qdd_test_ras_wait(int(extra_bytes), int(max_polls)), "qdd_test_ras_wait")


def measure_fma_peak(fp64: bool) -> float:
    """FMA throughput of the current GPU in TFLOP/s (FP64 or FP32)."""
    v = ctypes.c_double()
    _check(_lib.qdd_measure_fma_peak(int(bool(fp64)), ctypes.byref(v)), "qdd_measure_fma_peak")
    return v.value


def ras_field_noalloc(lat: Lattice, out: Field, inp: Field, rho: Field, v: Field, kappa: float, c_sw: float,
                      params: SolverParams) -> None:
    """out = K_RAS inp on internal fields without any device allocation (the
    scratch is a fixed array inside the library; see include/qdd.h)."""
    _check(_lib.qdd_ras_field_noalloc(lat.handle, out.handle, inp.handle, rho.handle, v.handle, float(kappa),
                                      float(c_sw), ctypes.byref(params)), "qdd_ras_field_noalloc")
