"""Plain FP64 CPU oracle (test infrastructure).

This package is the definition the GPU library is checked against.  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import it; the product package never does, and the two share no code.

The arithmetic lives in ``qdd_oracle.c`` (plain C, FP64, explicit 4x4 gamma
matrices and an explicit 12x12 clover per site), compiled here with gcc into
``liboracle.so`` and called through ctypes.  Each wrapper names the passage of
the paper it follows (Osaki & Ishikawa, Lattice 2010):

* ``dslash``       Eq. 1, the Wilson-clover operator D (Sec. 1, Sec. 5);
* ``clover``       the O(a) improvement term of Sec. 5 (c_SW);
* ``domain_*``     the Dirichlet-restricted operator and domain solve of Alg. 1;
* ``ras``          Alg. 1, phi = K_RAS eta (and the AS / SAP members of the
                   Schwarz family, Sec. 1 and Sec. 2);
* ``bicgstab``     the right-preconditioned Krylov solve of Eq. 3;
* ``solve``        the nested solver of Sec. 3 (FP64 defect correction);
* ``solve_nested`` the same with the paper's FP64 outer BiCGStab (Sec. 3).

Parity status of every function is pinned by ``tests/test_oracle_pins.py``.
``oracle/slab.py`` runs the paper's cluster decomposition (one x-slab domain
per rank, Sec. 4) on CPU ranks with these functions as its per-site pieces
(``tests/test_slab_ranks.py``).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qdd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class OraOp(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("bc", ctypes.c_int * 4),
                ("U", ctypes.c_void_p), ("A", ctypes.c_void_p), ("kappa", ctypes.c_double),
                ("csw", ctypes.c_double)]


class OraPrec(ctypes.Structure):
    _fields_ = [("use_ras", ctypes.c_int), ("block", ctypes.c_int * 4), ("s", ctypes.c_int),
                ("n_ras", ctypes.c_int), ("n_dominv", ctypes.c_int), ("dom_solver", ctypes.c_int),
                ("schwarz", ctypes.c_int)]


# Members of the Schwarz family (ora_prec.schwarz): RAS is Alg. 1; SAP is the
# multiplicative alternating procedure over a red/black block ordering; AS is
# the additive iteration without the restriction (overlaps summed).
SCHWARZ = {"ras": 0, "sap": 1, "as": 2}


class OraInfo(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("dv_count", ctypes.c_int), ("status", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I4 = ctypes.POINTER(ctypes.c_int)
            L.ora_set_threads.argtypes = [ctypes.c_int]
            L.ora_get_threads.restype = ctypes.c_int
            L.ora_gamma.argtypes = [ctypes.c_int, P]
            L.ora_field_strength.argtypes = [I4, P, ctypes.c_long, ctypes.c_int, ctypes.c_int, P]
            L.ora_clover.argtypes = [I4, P, ctypes.c_double, ctypes.c_double, P]
            L.ora_dslash.argtypes = [ctypes.POINTER(OraOp), P, P]
            L.ora_dslash_sites.argtypes = [ctypes.POINTER(OraOp), ctypes.c_long, P, P, P]
            L.ora_ndomains.argtypes = [I4, I4, ctypes.c_int]
            L.ora_ndomains.restype = ctypes.c_int
            L.ora_domain_sites.argtypes = [I4, I4, ctypes.c_int, ctypes.c_int, P, P]
            L.ora_domain_sites.restype = ctypes.c_long
            L.ora_domain_apply.argtypes = [ctypes.POINTER(OraOp), I4, ctypes.c_int, ctypes.c_int, P, P]
            L.ora_domain_apply.restype = ctypes.c_int
            L.ora_domain_solve.argtypes = [ctypes.POINTER(OraOp), ctypes.POINTER(OraPrec), ctypes.c_int, P, P]
            L.ora_domain_solve.restype = ctypes.c_int
            L.ora_ras.argtypes = [ctypes.POINTER(OraOp), ctypes.POINTER(OraPrec), P, P]
            L.ora_ras.restype = ctypes.c_int
            L.ora_bicgstab.argtypes = [ctypes.POINTER(OraOp), ctypes.POINTER(OraPrec), P, P,
                                       ctypes.c_double, ctypes.c_int, I4, I4]
            L.ora_bicgstab.restype = ctypes.c_int
            L.ora_solve.argtypes = [ctypes.POINTER(OraOp), ctypes.POINTER(OraPrec), ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P,
                                    ctypes.POINTER(OraInfo)]
            L.ora_solve.restype = ctypes.c_int
            L.ora_solve_nested.argtypes = L.ora_solve.argtypes
            L.ora_solve_nested.restype = ctypes.c_int
            L.ora_true_residual.argtypes = [ctypes.POINTER(OraOp), P, P]
            L.ora_true_residual.restype = ctypes.c_double
            _lib = L
    return _lib


def _i4(v):
    return (ctypes.c_int * 4)(*[int(a) for a in v])


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def get_threads() -> int:
    return lib().ora_get_threads()


def gamma(mu: int) -> np.ndarray:
    """gamma_{mu+1} for mu = 0..3 (x, y, z, t) and gamma_5 for mu = 4."""
    g = np.zeros((4, 4), dtype=np.complex128)
    lib().ora_gamma(mu, g.ctypes.data)
    return g


def field_strength(dims, U, site: int, mu: int, nu: int) -> np.ndarray:
    U, pu = _c(U)
    F = np.zeros((3, 3), dtype=np.complex128)
    lib().ora_field_strength(_i4(dims), pu, site, mu, nu, F.ctypes.data)
    return F


def clover(dims, U, kappa: float, c_sw: float) -> np.ndarray:
    """A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) Fhat_{mu nu}(x), [V][12][12]."""
    U, pu = _c(U)
    V = int(np.prod(dims))
    A = np.empty((V, 12, 12), dtype=np.complex128)
    lib().ora_clover(_i4(dims), pu, float(kappa), float(c_sw), A.ctypes.data)
    return A


class Op:
    """The Wilson-clover operator D = A - kappa H for one gauge field (Eq. 1)."""

    def __init__(self, dims, bc, U, kappa: float, c_sw: float, A=None, store_clover: bool = True):
        """``store_clover=False`` keeps no [V][12][12] array and rebuilds A(x)
        from the links at every use (for sampled checks on large lattices)."""
        self.dims = tuple(int(d) for d in dims)
        self.bc = tuple(int(b) for b in bc)
        self.V = int(np.prod(self.dims))
        self.U = np.ascontiguousarray(U, dtype=np.complex128).reshape(self.V, 4, 3, 3)
        self.kappa = float(kappa)
        self.c_sw = float(c_sw)
        if A is not None:
            self.A = np.ascontiguousarray(A, dtype=np.complex128)
        elif store_clover:
            self.A = clover(self.dims, self.U, kappa, c_sw)
        else:
            self.A = None
        self._s = OraOp(_i4(self.dims), _i4(self.bc), self.U.ctypes.data,
                        None if self.A is None else self.A.ctypes.data, self.kappa, self.c_sw)

    def shape(self):
        return (self.V, 4, 3)

    def dslash(self, psi) -> np.ndarray:
        psi, pp = _c(psi)
        out = np.empty(self.shape(), dtype=np.complex128)
        lib().ora_dslash(ctypes.byref(self._s), pp, out.ctypes.data)
        return out

    def dslash_sites(self, psi, sites) -> np.ndarray:
        """(D psi) evaluated at the given sites only, [len(sites)][4][3]."""
        psi, pp = _c(psi)
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        out = np.empty((sites.size, 4, 3), dtype=np.complex128)
        lib().ora_dslash_sites(ctypes.byref(self._s), sites.size, sites.ctypes.data, pp, out.ctypes.data)
        return out

    # -- domains (Alg. 1 lines 4-6) ------------------------------------
    def ndomains(self, block, s: int) -> int:
        return lib().ora_ndomains(_i4(self.dims), _i4(block), int(s))

    def domain_sites(self, block, s: int, dom: int):
        n = lib().ora_domain_sites(_i4(self.dims), _i4(block), int(s), int(dom), None, None)
        if n < 0:
            raise ValueError("invalid blocking")
        sites = np.empty(n, dtype=np.int64)
        bulk = np.empty(n, dtype=np.int32)
        lib().ora_domain_sites(_i4(self.dims), _i4(block), int(s), int(dom), sites.ctypes.data, bulk.ctypes.data)
        return sites, bulk.astype(bool)

    def domain_apply(self, block, s: int, dom: int, vloc) -> np.ndarray:
        vloc, pv = _c(vloc)
        out = np.empty_like(vloc)
        if lib().ora_domain_apply(ctypes.byref(self._s), _i4(block), int(s), int(dom), pv, out.ctypes.data):
            raise ValueError("invalid blocking")
        return out

    def domain_solve(self, block, s: int, dom: int, rloc, n_dominv: int = 4, exact: bool = False):
        rloc, pr = _c(rloc)
        out = np.empty_like(rloc)
        p = prec(True, block, s, 1, n_dominv, exact)
        if lib().ora_domain_solve(ctypes.byref(self._s), ctypes.byref(p), int(dom), pr, out.ctypes.data):
            raise ValueError("invalid blocking")
        return out

    # -- Alg. 1, Eq. 3, Sec. 3 ------------------------------------------
    def ras(self, eta, block, s: int = 0, n_ras: int = 3, n_dominv: int = 4, exact: bool = False,
            schwarz: str = "ras"):
        """NRAS cycles of the Schwarz iteration from phi = 0 (Alg. 1 for
        schwarz="ras"; "sap" and "as" are the multiplicative and the plain
        additive members of the family, Sec. 1 and Sec. 2)."""
        eta, pe = _c(eta)
        out = np.empty(self.shape(), dtype=np.complex128)
        p = prec(True, block, s, n_ras, n_dominv, exact, schwarz)
        if lib().ora_ras(ctypes.byref(self._s), ctypes.byref(p), pe, out.ctypes.data):
            raise ValueError("invalid blocking")
        return out

    def bicgstab(self, b, tol: float, maxit: int = 10000, ras=None):
        """One right-preconditioned BiCGStab solve; ``ras`` is None or a dict
        of prec() keyword arguments.  Returns (x, status, iters, dv_count)."""
        b, pb = _c(b)
        x = np.zeros(self.shape(), dtype=np.complex128)
        p = prec(False) if ras is None else prec(True, **ras)
        it = ctypes.c_int(0)
        dv = ctypes.c_int(0)
        st = lib().ora_bicgstab(ctypes.byref(self._s), ctypes.byref(p), pb, x.ctypes.data,
                                float(tol), int(maxit), ctypes.byref(it), ctypes.byref(dv))
        return x, st, it.value, dv.value

    def solve(self, eta, tol: float, inner_tol: float = None, ras=None, max_inner: int = 100000,
              max_outer: int = 100):
        """Nested solve with FP64 defect correction.  With ``ras=None`` and
        ``inner_tol=None`` this is the plain BiCGStab continued from the true
        residual.  Returns (phi, info dict)."""
        eta, pe = _c(eta)
        phi = np.zeros(self.shape(), dtype=np.complex128)
        p = prec(False) if ras is None else prec(True, **ras)
        info = OraInfo()
        lib().ora_solve(ctypes.byref(self._s), ctypes.byref(p), float(tol if inner_tol is None else inner_tol),
                        int(max_inner), int(max_outer), float(tol), pe, phi.ctypes.data, ctypes.byref(info))
        return phi, {k: getattr(info, k) for k, _ in OraInfo._fields_}

    def solve_nested(self, eta, tol: float, inner_tol: float = 1e-3, ras=None, max_inner: int = 100000,
                     max_outer: int = 1000):
        """The paper's nested solver (Sec. 3): FP64 outer BiCGStab with the
        inner BiCGStab (right-preconditioned by K when ``ras`` is a dict of
        prec() arguments) as a flexible preconditioner, restarted from the
        true residual until it meets tol.  Returns (phi, info dict);
        outer_iters counts outer BiCGStab iterations."""
        eta, pe = _c(eta)
        phi = np.zeros(self.shape(), dtype=np.complex128)
        p = prec(False) if ras is None else prec(True, **ras)
        info = OraInfo()
        lib().ora_solve_nested(ctypes.byref(self._s), ctypes.byref(p), float(inner_tol), int(max_inner),
                               int(max_outer), float(tol), pe, phi.ctypes.data, ctypes.byref(info))
        return phi, {k: getattr(info, k) for k, _ in OraInfo._fields_}

    def true_residual(self, eta, phi) -> float:
        """|eta - D phi| / |eta| (Sec. 5 stopping rule)."""
        eta, pe = _c(eta)
        phi, pp = _c(phi)
        return lib().ora_true_residual(ctypes.byref(self._s), pe, pp)


def prec(use_ras: bool, block=(4, 4, 4, 4), s: int = 0, n_ras: int = 3, n_dominv: int = 4,
         exact: bool = False, schwarz: str = "ras") -> OraPrec:
    return OraPrec(int(bool(use_ras)), _i4(block), int(s), int(n_ras), int(n_dominv), int(bool(exact)),
                   SCHWARZ[schwarz])
