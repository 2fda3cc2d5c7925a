"""CPU oracle for the KKT refactor / solve / refine path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never touches it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, single thread; see its
header for which passage of the paper each routine follows). This module
compiles it with gcc on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, no FMA contraction so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.ora_ruiz.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_int, _f64p]
        lib.ora_ruiz.restype = C.c_int
        lib.ora_min_degree.argtypes = [C.c_int, _i32p, _i32p, _i32p]
        lib.ora_min_degree.restype = C.c_int
        lib.ora_lu.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, C.c_void_p, C.c_double, C.c_double]
        lib.ora_lu.restype = C.c_void_p
        lib.ora_lu_free.argtypes = [C.c_void_p]
        for f in ("ora_lu_n", "ora_lu_nnz_l", "ora_lu_nnz_u", "ora_lu_n_perturbed", "ora_lu_n_offdiag"):
            getattr(lib, f).argtypes = [C.c_void_p]
            getattr(lib, f).restype = C.c_int
        lib.ora_lu_export.argtypes = [C.c_void_p, _i32p, _i32p, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p]
        lib.ora_solve.argtypes = [C.c_void_p, _f64p, _f64p]
        lib.ora_solve_scaled.argtypes = [C.c_void_p, _f64p, _f64p, _f64p]
        lib.ora_spmv_resid.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
        lib.ora_matrix_norm_inf.argtypes = [C.c_int, _i32p, _i32p, _f64p]
        lib.ora_matrix_norm_inf.restype = C.c_double
        lib.ora_backward_error.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p]
        lib.ora_backward_error.restype = C.c_double
        lib.ora_fgmres.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_void_p, _f64p, _f64p, _f64p,
                                   C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double)]
        lib.ora_fgmres.restype = C.c_int
        lib.ora_lu_error_bound.argtypes = [C.c_void_p, _i32p, _i32p, _f64p, C.c_double, C.c_double, _f64p, _f64p]
        _lib = lib
    return _lib


def _csr(rowptr, colidx, vals=None):
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    if vals is None:
        return rp, ci
    return rp, ci, np.ascontiguousarray(vals, dtype=np.float64)


def ruiz(rowptr, colidx, vals, iters: int = 10):
    """Power-of-two symmetric Ruiz scaling d (so that D A D is equilibrated)."""
    rp, ci, v = _csr(rowptr, colidx, vals)
    n = rp.size - 1
    d = np.empty(n)
    it = _load().ora_ruiz(n, rp, ci, v, int(iters), d)
    return d, it


def scale(rowptr, colidx, vals, d):
    """D A D in the CSR order of A."""
    rp, ci, v = _csr(rowptr, colidx, vals)
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    return d[rows] * v * d[ci]


def min_degree(rowptr, colidx):
    rp, ci = _csr(rowptr, colidx)
    n = rp.size - 1
    q = np.empty(n, dtype=np.int32)
    _load().ora_min_degree(n, rp, ci, q)
    return q


@dataclass
class Factors:
    """L (unit, diagonal not stored) and U (diagonal last) of P A Q in CSC over steps."""
    p: np.ndarray
    q: np.ndarray
    Lp: np.ndarray
    Li: np.ndarray
    Lx: np.ndarray
    Up: np.ndarray
    Ui: np.ndarray
    Ux: np.ndarray
    n_perturbed: int
    n_offdiag: int
    handle: "LU"

    @property
    def n(self):
        return self.p.size


class LU:
    """Owns an oracle factorization handle."""

    def __init__(self, rowptr, colidx, scaled_vals, q, p=None, tau=0.0, pivot_floor=0.0):
        lib = _load()
        rp, ci, v = _csr(rowptr, colidx, scaled_vals)
        self.n = n = rp.size - 1
        qq = np.ascontiguousarray(q, dtype=np.int32)
        self._keep = (rp, ci, v, qq)
        pp = None
        if p is not None:
            pp = np.ascontiguousarray(p, dtype=np.int32)
            self._keep = self._keep + (pp,)
        self.h = lib.ora_lu(n, rp, ci, v, qq, pp.ctypes.data if pp is not None else None,
                            float(tau), float(pivot_floor))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ora_lu_free(self.h)
            self.h = None

    def factors(self) -> Factors:
        lib = _load()
        n = self.n
        nl, nu = lib.ora_lu_nnz_l(self.h), lib.ora_lu_nnz_u(self.h)
        p, q = np.empty(n, np.int32), np.empty(n, np.int32)
        Lp, Up = np.empty(n + 1, np.int32), np.empty(n + 1, np.int32)
        Li, Lx = np.empty(max(nl, 1), np.int32), np.empty(max(nl, 1))
        Ui, Ux = np.empty(max(nu, 1), np.int32), np.empty(max(nu, 1))
        lib.ora_lu_export(self.h, p, q, Lp, Li, Lx, Up, Ui, Ux)
        return Factors(p, q, Lp, Li[:nl], Lx[:nl], Up, Ui[:nu], Ux[:nu],
                       lib.ora_lu_n_perturbed(self.h), lib.ora_lu_n_offdiag(self.h), self)

    def error_bound(self, rowptr, colidx, scaled_vals, unit=2.0 ** -53, pivot_floor=0.0):
        """First-order running error bounds (eL, eU) aligned with Lx / Ux for a
        computation of these factors in a format of unit roundoff `unit`."""
        rp, ci, v = _csr(rowptr, colidx, scaled_vals)
        lib = _load()
        nl, nu = lib.ora_lu_nnz_l(self.h), lib.ora_lu_nnz_u(self.h)
        eL, eU = np.zeros(max(nl, 1)), np.zeros(max(nu, 1))
        lib.ora_lu_error_bound(self.h, rp, ci, v, float(unit), float(pivot_floor), eL, eU)
        return eL[:nl], eU[:nu]

    def solve(self, c):
        z = np.empty(self.n)
        _load().ora_solve(self.h, np.ascontiguousarray(c, dtype=np.float64), z)
        return z

    def solve_scaled(self, d, b):
        x = np.empty(self.n)
        _load().ora_solve_scaled(self.h, np.ascontiguousarray(d, np.float64),
                                 np.ascontiguousarray(b, np.float64), x)
        return x


def jacobi_precondition(f: Factors, d, b, sweeps: int):
    """Approximate solve of K x = b by Jacobi sweeps with the factors of the
    scaled, permuted matrix (Sec. V proposes iterative triangular solves in
    place of the exact ones), written as the plain definition:
        c = P D b;   y_0 = 0,  y_{s+1} = c - (L - I) y_s;
        x_0 = 0,  x_{s+1} = diag(U)^{-1} (y - (U - diag(U)) x_s);
        result = D Q x.
    f: factors of P (D K D) Q (L unit lower with its diagonal not stored, U
    with its diagonal last in each column), d: the equilibration factors."""
    import scipy.sparse as sp
    n = f.n
    Ls = sp.csc_matrix((f.Lx, f.Li, f.Lp), shape=(n, n))        # L - I
    U = sp.csc_matrix((f.Ux, f.Ui, f.Up), shape=(n, n))
    du = U.diagonal()
    Us = (U - sp.diags(du)).tocsr()
    c = (np.asarray(d) * np.asarray(b))[f.p]
    y = np.zeros(n)
    for _ in range(sweeps):
        y = c - Ls @ y
    x = np.zeros(n)
    for _ in range(sweeps):
        x = (y - Us @ x) / du
    z = np.empty(n)
    z[f.q] = x
    return np.asarray(d) * z


def _block_parts(f: Factors, block_of):
    """(L_D, L_O, U_D, U_O) of block_jacobi_precondition, CSR in pivot order."""
    import scipy.sparse as sp
    n = f.n
    blk = np.asarray(block_of)[f.q]
    Ls = sp.csc_matrix((f.Lx, f.Li, f.Lp), shape=(n, n)).tocoo()      # L - I
    U = sp.csc_matrix((f.Ux, f.Ui, f.Up), shape=(n, n)).tocoo()
    same_l = blk[Ls.row] == blk[Ls.col]
    same_u = blk[U.row] == blk[U.col]
    LD = (sp.eye(n, format="csr") + sp.csr_matrix((Ls.data[same_l], (Ls.row[same_l], Ls.col[same_l])),
                                                   shape=(n, n))).tocsr()
    LO = sp.csr_matrix((Ls.data[~same_l], (Ls.row[~same_l], Ls.col[~same_l])), shape=(n, n))
    UD = sp.csr_matrix((U.data[same_u], (U.row[same_u], U.col[same_u])), shape=(n, n))
    UO = sp.csr_matrix((U.data[~same_u], (U.row[~same_u], U.col[~same_u])), shape=(n, n))
    return LD, LO, UD, UO


def block_jacobi_precondition(f: Factors, d, b, sweeps: int, block_of):
    """Approximate solve of K x = b by block-Jacobi sweeps with the factors,
    Gauss-Seidel (an exact substitution) within each block: the iterative
    triangular solves of Sec. V with the pivots grouped in blocks. With L_D,
    U_D the parts of L and U whose row and column lie in one block and L_O =
    L - L_D, U_O = U - U_D, written as the plain definition:
        c = P D b;   y_0 = 0,  y_{s+1} = L_D^{-1} (c - L_O y_s);
        x_0 = 0,  x_{s+1} = U_D^{-1} (y - U_O x_s);
        result = D Q x.
    block_of: the block of every unknown, in the original numbering (pivot
    position i belongs to the block of unknown q[i]). Singleton blocks give
    the point-Jacobi sweeps above; one block gives the exact solve."""
    import scipy.sparse.linalg as spla
    n = f.n
    LD, LO, UD, UO = _block_parts(f, block_of)
    c = (np.asarray(d) * np.asarray(b))[f.p]
    y = np.zeros(n)
    for _ in range(sweeps):
        y = spla.spsolve_triangular(LD, c - LO @ y, lower=True, unit_diagonal=True)
    x = np.zeros(n)
    for _ in range(sweeps):
        x = spla.spsolve_triangular(UD, y - UO @ x, lower=False)
    z = np.empty(n)
    z[f.q] = x
    return np.asarray(d) * z


def spmv_resid(rowptr, colidx, vals, x, b):
    rp, ci, v = _csr(rowptr, colidx, vals)
    r = np.empty(rp.size - 1)
    _load().ora_spmv_resid(rp.size - 1, rp, ci, v, np.ascontiguousarray(x, np.float64),
                           np.ascontiguousarray(b, np.float64), r)
    return r


def matrix_norm_inf(rowptr, colidx, vals):
    rp, ci, v = _csr(rowptr, colidx, vals)
    return _load().ora_matrix_norm_inf(rp.size - 1, rp, ci, v)


def backward_error(rowptr, colidx, vals, x, b):
    rp, ci, v = _csr(rowptr, colidx, vals)
    return _load().ora_backward_error(rp.size - 1, rp, ci, v, np.ascontiguousarray(x, np.float64),
                                      np.ascontiguousarray(b, np.float64))


def fgmres(rowptr, colidx, vals, lu: LU, d, b, restart=30, max_cycles=10, tol=1e-10):
    """FGMRES(restart) refinement; returns (x, inner iterations, omega)."""
    rp, ci, v = _csr(rowptr, colidx, vals)
    x = np.empty(rp.size - 1)
    om = C.c_double(0.0)
    it = _load().ora_fgmres(rp.size - 1, rp, ci, v, lu.h, np.ascontiguousarray(d, np.float64),
                            np.ascontiguousarray(b, np.float64), x, int(restart), int(max_cycles),
                            float(tol), C.byref(om))
    return x, it, om.value


# ------------------------------------------------------------ composite use

@dataclass
class Analysis:
    """Oracle-side analysis of the first matrix: scaling, ordering, pivot rows."""
    d0: np.ndarray
    q: np.ndarray
    p: np.ndarray
    n_offdiag: int


def analyze(rowptr, colidx, vals, tau=0.0, ruiz_iters=10, pivot_eps=1e-14):
    """Alg. 1 first system: scale, order, factor with threshold pivoting, keep P and Q."""
    d0, _ = ruiz(rowptr, colidx, vals, ruiz_iters)
    sv = scale(rowptr, colidx, vals, d0)
    q = min_degree(rowptr, colidx)
    floor = pivot_eps * np.abs(sv).max()
    f = LU(rowptr, colidx, sv, q, None, tau, floor).factors()
    return Analysis(d0, q, f.p.copy(), f.n_offdiag)


def refactor(rowptr, colidx, vals, an: Analysis, ruiz_iters=10, pivot_eps=1e-14):
    """Alg. 1 refactor step for a later matrix: rescale, frozen P and Q, static pivots."""
    d, _ = ruiz(rowptr, colidx, vals, ruiz_iters)
    sv = scale(rowptr, colidx, vals, d)
    floor = pivot_eps * np.abs(sv).max()
    lu = LU(rowptr, colidx, sv, an.q, an.p, 0.0, floor)
    return lu, d, sv
