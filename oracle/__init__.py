"""Oracle: a plain, slow, obviously correct CPU statement of what the solver computes.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference arm may import this package. The product package
(paper_1511_07174_gb300) never imports it, and it never imports the product.

Contents
  * gbla_oracle.c (ctypes, FP64): GEPP, Cholesky, substitution, backward
    error, gradient of solve, pivot-gap diagnostic -- paper section 2.
  * gmres.py (numpy, FP64): restarted GMRES with modified Gram-Schmidt and
    Givens rotations (paper section 2) and the GMRES-based iterative
    refinement loop built on it.
  * mixed.py (numpy): the low-precision blocked LU whose trailing update uses
    operands rounded to FP32 / TF32 / BF16 / FP16 with power-of-two scaling.

Every array argument is a float64 numpy array in column-major (Fortran) order.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_getrf_steps.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ip, ctypes.c_int]
        L.oracle_getrf.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ip]
        L.oracle_potrf.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip]
        L.oracle_getrs.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip, dp, ctypes.c_int]
        L.oracle_potrs.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int]
        L.oracle_backward_error.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp,
                                            ctypes.c_int, dp, ctypes.c_int, dp]
        L.oracle_solve_grad.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int,
                                        dp, ctypes.c_int, dp, dp]
        L.oracle_min_pivot_gap.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int]
        L.oracle_min_pivot_gap.restype = ctypes.c_double
        _lib = L
    return _lib


def _f64(a):
    a = np.asfortranarray(np.asarray(a, dtype=np.float64))
    return a


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _as2d(b):
    b = np.asarray(b, dtype=np.float64)
    return b.reshape(-1, 1) if b.ndim == 1 else b


def getrf(A, ksteps=None):
    """P A = L U by GEPP. Returns (LU packed, ipiv int32 1-based, info)."""
    LU = _f64(A).copy(order="F")
    n = LU.shape[0]
    ipiv = np.zeros(max(n, 1), dtype=np.int32)
    info = np.zeros(1, dtype=np.int32)
    k = n if ksteps is None else int(ksteps)
    rc = lib().oracle_getrf_steps(n, _dp(LU), max(n, 1), _ip(ipiv), _ip(info), k)
    assert rc == 0
    return LU, ipiv[:n], int(info[0])


def potrf(A):
    """A = L L^t (lower). Returns (matrix with L in the lower triangle, info)."""
    L = _f64(A).copy(order="F")
    n = L.shape[0]
    info = np.zeros(1, dtype=np.int32)
    rc = lib().oracle_potrf(n, _dp(L), max(n, 1), _ip(info))
    assert rc == 0
    return L, int(info[0])


def getrs(LU, ipiv, B):
    LU = _f64(LU)
    X = np.asfortranarray(_as2d(B).copy())
    n, nrhs = X.shape
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    rc = lib().oracle_getrs(n, nrhs, _dp(LU), max(n, 1), _ip(piv), _dp(X), max(n, 1))
    assert rc == 0
    return X


def potrs(L, B):
    L = _f64(L)
    X = np.asfortranarray(_as2d(B).copy())
    n, nrhs = X.shape
    rc = lib().oracle_potrs(n, nrhs, _dp(L), max(n, 1), _dp(X), max(n, 1))
    assert rc == 0
    return X


def backward_error(A, X, B):
    """Per-column ||b - A x||_inf / (||A||_inf ||x||_inf) in plain FP64."""
    A = _f64(A)
    X = np.asfortranarray(_as2d(X))
    B = np.asfortranarray(_as2d(B))
    n, nrhs = X.shape
    beta = np.zeros(max(nrhs, 1), dtype=np.float64)
    rc = lib().oracle_backward_error(n, nrhs, _dp(A), max(n, 1), _dp(X), max(n, 1), _dp(B),
                                     max(n, 1), _dp(beta))
    assert rc == 0
    return beta[:nrhs]


def solve_grad(A, X, G):
    """(gA, gB) for x = A^{-1} b with upstream gradient G: gB = A^{-t} G, gA = -gB X^t."""
    A = _f64(A)
    X = np.asfortranarray(_as2d(X))
    G = np.asfortranarray(_as2d(G))
    n, nrhs = X.shape
    gA = np.zeros((n, n), dtype=np.float64, order="F")
    gB = np.zeros((n, nrhs), dtype=np.float64, order="F")
    info = lib().oracle_solve_grad(n, nrhs, _dp(A), max(n, 1), _dp(X), max(n, 1), _dp(G),
                                   max(n, 1), _dp(gA), _dp(gB))
    assert info == 0, info
    return gA, gB


def min_pivot_gap(A, ksteps=None):
    A = _f64(A)
    n = A.shape[0]
    return float(lib().oracle_min_pivot_gap(n, _dp(A), max(n, 1), n if ksteps is None else int(ksteps)))


def unpack_lu(LU):
    """Split packed LU into (L unit lower, U upper)."""
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    return L, U


def perm_from_ipiv(ipiv, n):
    """Row order p such that (P A)[i] = A[p[i]] for the sequential swaps ipiv."""
    p = np.arange(n)
    for j in range(len(ipiv)):
        k = int(ipiv[j]) - 1
        p[j], p[k] = p[k], p[j]
    return p
