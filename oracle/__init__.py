"""CPU oracle for the DD / QD matrix products (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It is built from ``oracle.cpp`` with g++ and is
independent of the CUDA library: the two share no source, header or helper.

Every function follows the paper (Kouya 2015) as cited in ``oracle.cpp``:
Section 2 Eq. 1 for the Simple product, Section 4 for the LU tests; the DD/QD
operation sequences are the published error-free transformations named
there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp into _build/liboracle.so (a few seconds)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        d, i64, vp, ci = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        L.orc_two_sum.argtypes = [d, d, vp]
        L.orc_two_prod.argtypes = [d, d, vp]
        for f in (L.orc_dd_mul, L.orc_dd_add, L.orc_qd_mul, L.orc_qd_add):
            f.argtypes = [vp, vp, vp]
        L.orc_renorm.argtypes = [vp, ci, vp]
        L.orc_exact_dot.argtypes = [i64, vp, vp, vp]
        L.orc_exact_dot.restype = d
        L.orc_dd_gemm_simple.argtypes = [i64, i64, i64, vp, vp, i64, vp, vp, i64, vp, vp, i64, ci, ci]
        L.orc_qd_gemm_simple.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, ci, ci]
        L.orc_gemm_error.argtypes = [ci, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, ci,
                                     i64, vp, vp, vp, ci]
        L.orc_gemm_exact.argtypes = [ci, i64, i64, i64, vp, i64, vp, i64, vp, ci]
        L.orc_dd_residual.argtypes = [i64, i64, vp, vp, i64, vp, vp, i64, vp, vp, i64, vp, ci]
        L.orc_dd_getrf.argtypes = [i64, vp, vp, i64, vp, ci]
        L.orc_dd_getrf.restype = ci
        L.orc_residual.argtypes = [ci, i64, i64, vp, i64, vp, i64, vp, i64, vp, ci]
        L.orc_qd_getrf.argtypes = [i64, vp, i64, vp, ci]
        L.orc_qd_getrf.restype = ci
        L.orc_qd_div.argtypes = [vp, vp, vp]
        _lib = L
    return _lib


def threads() -> int:
    return max(1, os.cpu_count() or 1)


def _p(a: np.ndarray) -> int:
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data


def _planes(M: np.ndarray):
    arr = (ctypes.c_void_p * M.shape[0])(*[M[k].ctypes.data for k in range(M.shape[0])])
    return arr


# --------------------------------------------------------------- scalars ----
def two_sum(a: float, b: float):
    out = np.zeros(2)
    lib().orc_two_sum(a, b, _p(out))
    return out[0], out[1]


def two_prod(a: float, b: float):
    out = np.zeros(2)
    lib().orc_two_prod(a, b, _p(out))
    return out[0], out[1]


def _binop(fn, a, b, k):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(k)
    fn(_p(a), _p(b), _p(out))
    return out


def dd_mul(a, b):
    return _binop(lib().orc_dd_mul, a, b, 2)


def dd_add(a, b):
    return _binop(lib().orc_dd_add, a, b, 2)


def qd_mul(a, b):
    return _binop(lib().orc_qd_mul, a, b, 4)


def qd_add(a, b):
    return _binop(lib().orc_qd_add, a, b, 4)


def qd_div(a, b):
    return _binop(lib().orc_qd_div, a, b, 4)


def renorm(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_renorm(_p(x), len(x), _p(out))
    return out


def exact_dot(x, y=None, neg=None) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    yp = None if y is None else _p(np.ascontiguousarray(y, dtype=np.float64))
    ng = None if neg is None else np.ascontiguousarray(neg, dtype=np.int32)
    return lib().orc_exact_dot(len(x), _p(x), yp, None if ng is None else ng.ctypes.data)


# ----------------------------------------------------------------- GEMMs ----
MODES = {"set": 0, "add": 1, "sub": 2}


def gemm_simple(A: np.ndarray, B: np.ndarray, C0: np.ndarray | None = None,
                mode: str = "set", nthreads: int | None = None) -> np.ndarray:
    """Eq. 1 Simple product in DD (2 planes) or QD (4 planes).

    A: (limbs, m, l), B: (limbs, l, n); returns C (limbs, m, n).
    mode 'add' / 'sub' start from C0 and add / subtract A B.
    """
    limbs, m, l = A.shape
    n = B.shape[2]
    assert B.shape == (limbs, l, n)
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    C = np.zeros((limbs, m, n)) if C0 is None else np.array(C0, dtype=np.float64, order="C")
    nt = nthreads or threads()
    md = MODES[mode]
    if limbs == 2:
        rc = lib().orc_dd_gemm_simple(m, l, n, _p(A[0]), _p(A[1]), max(l, 1),
                                      _p(B[0]), _p(B[1]), max(n, 1),
                                      C[0].ctypes.data, C[1].ctypes.data, max(n, 1), md, nt)
    elif limbs == 4:
        rc = lib().orc_qd_gemm_simple(m, l, n, _planes(A), max(l, 1), _planes(B), max(n, 1),
                                      _planes(C), max(n, 1), md, nt)
    else:
        raise ValueError("limbs must be 2 or 4")
    assert rc == 0
    return C


def gemm_error(A, B, C, C0=None, mode: str = "set", rows=None, cols=None,
               nthreads: int | None = None) -> np.ndarray:
    """Exact error (exact - computed) per entry, rounded to double.

    With rows/cols given, only those entries; else all entries (m, n).
    """
    limbs, m, l = A.shape
    n = B.shape[2]
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    C = np.ascontiguousarray(C)
    c0 = None if C0 is None else _planes(np.ascontiguousarray(C0))
    if rows is None:
        err = np.zeros(m * n)
        cnt, rp, cp = -1, None, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        err = np.zeros(len(rows))
        cnt, rp, cp = len(rows), rows.ctypes.data, cols.ctypes.data
    rc = lib().orc_gemm_error(limbs, m, l, n, _planes(A), max(l, 1), _planes(B), max(n, 1),
                              _planes(C), max(n, 1), c0, MODES[mode], cnt, rp, cp,
                              _p(err), nthreads or threads())
    assert rc == 0
    return err.reshape(m, n) if rows is None else err


def gemm_exact(A, B, nthreads: int | None = None) -> np.ndarray:
    """Exact A B per entry rounded to the nearest double."""
    limbs, m, l = A.shape
    n = B.shape[2]
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    out = np.zeros(m * n)
    lib().orc_gemm_exact(limbs, m, l, n, _planes(A), max(l, 1), _planes(B), max(n, 1),
                         _p(out), nthreads or threads())
    return out.reshape(m, n)


def dd_residual(A, X, Bv, nthreads: int | None = None) -> np.ndarray:
    """Exact b - A x per entry (Section 4, Eq. 2), rounded to double."""
    n = A.shape[1]
    nrhs = X.shape[2]
    A, X, Bv = (np.ascontiguousarray(v) for v in (A, X, Bv))
    r = np.zeros(n * nrhs)
    lib().orc_dd_residual(n, nrhs, _p(A[0]), _p(A[1]), n, _p(X[0]), _p(X[1]), nrhs,
                          _p(Bv[0]), _p(Bv[1]), nrhs, _p(r), nthreads or threads())
    return r.reshape(n, nrhs)


def dd_getrf(A, pivot: bool = True):
    """Unblocked DD LU in place on a copy; returns (LU, ipiv, info)."""
    n = A.shape[1]
    LU = np.array(A, dtype=np.float64, order="C")
    ipiv = np.zeros(n, dtype=np.int64)
    info = lib().orc_dd_getrf(n, LU[0].ctypes.data, LU[1].ctypes.data, n, ipiv.ctypes.data,
                              1 if pivot else 0)
    return LU, ipiv, info


def residual(A, X, Bv, nthreads: int | None = None) -> np.ndarray:
    """Exact b - A x per entry for DD or QD operands (Section 4, Eq. 2)."""
    limbs, n = A.shape[0], A.shape[1]
    nrhs = X.shape[2]
    A, X, Bv = (np.ascontiguousarray(v, dtype=np.float64) for v in (A, X, Bv))
    r = np.zeros(n * nrhs)
    lib().orc_residual(limbs, n, nrhs, _planes(A), n, _planes(X), nrhs, _planes(Bv), nrhs, _p(r),
                       nthreads or threads())
    return r.reshape(n, nrhs)


def qd_getrf(A, pivot: bool = True):
    """Unblocked QD LU in place on a copy; returns (LU, ipiv, info)."""
    n = A.shape[1]
    LU = np.array(A, dtype=np.float64, order="C")
    ipiv = np.zeros(n, dtype=np.int64)
    info = lib().orc_qd_getrf(n, _planes(LU), n, ipiv.ctypes.data, 1 if pivot else 0)
    return LU, ipiv, info


def normwise(err: np.ndarray, A: np.ndarray, B: np.ndarray) -> float:
    """||C - C^||_F / (||A||_F ||B||_F), norms of A and B from leading limbs."""
    return float(np.linalg.norm(err) / (np.linalg.norm(A[0]) * np.linalg.norm(B[0])))
