"""Oracle for the INT8-slice DD product (test infrastructure only).

A plain restatement, in Python integers and numpy int64, of the splitting
scheme of Ozaki, Ogita and Oishi (2012) in the integer form the CUDA library
documents for its DDG_OZAKI algorithm, step by step:

1. per row i of A (column j of B): f_i = the largest biased exponent field of
   the leading limbs (at least 1), so every |a_ik| < 2^(f_i - 1022);
2. X_ik = round-half-up of a_ik 2^(T - e_i) with T = 6 + 7 (s - 1) and
   e_i = f_i - 1022, where each limb's contribution is first truncated toward
   zero at 2^-64 units;
3. balanced base-128 digits: X = sum_p d_p 128^(s - p), d_p in [-64, 63]
   for p >= 2 (least significant first) and d_1 the remainder;
4. D_r = sum_{p + q = r} alpha^(p) beta^(q) for r = 2 .. s + 1 (int64 GEMMs);
5. V = sum_r D_r 2^(7 (s + 1 - r)) exactly, c = V 2^(e_i + e_j - T - 6);
   rounded to DD as: hi = leading 53 bits of |V| (truncated), lo = next 53
   bits (truncated), signs applied, then TwoSum(hi, lo); to QD as four such
   53-bit pieces, renormalised (the oracle's VecSum + compaction).

Slow and obviously exact; for small matrices.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import dd_add, qd_add, renorm


def exp_field(x: float) -> int:
    if x == 0.0 or not math.isfinite(x):
        return 0
    b = np.float64(x).view(np.uint64)
    return int((int(b) >> 52) & 0x7FF)


def row_fields(M0: np.ndarray, axis: int) -> np.ndarray:
    """Largest exponent field (>= 1) along `axis` of the leading-limb plane."""
    f = np.vectorize(exp_field, otypes=[np.int64])(M0)
    return np.maximum(f.max(axis=axis), 1)


def to_integer(limbs, field: int, s: int) -> int:
    T = 6 + 7 * (s - 1)
    e = field - 1022
    acc = 0
    for limb in limbs:
        v = Fraction(float(limb)) * Fraction(2) ** (T - e + 64)
        acc += int(v)  # truncation toward zero at 2^-64 units
    return (acc + (1 << 63)) >> 64


def digits(X: int, s: int) -> list:
    """Balanced base-128 digits, most significant first (length s)."""
    out = [0] * s
    for p in range(s, 1, -1):
        d = X & 127
        if d >= 64:
            d -= 128
        out[p - 1] = d
        X = (X - d) >> 7
    out[0] = X
    return out


def split(M: np.ndarray, s: int, by_row: bool):
    """Slices (s, rows, cols) int64 and the fields per row (A) / column (B)."""
    _, rows, cols = M.shape
    f = row_fields(M[0], axis=1 if by_row else 0)
    S = np.zeros((s, rows, cols), dtype=np.int64)
    for i in range(rows):
        for k in range(cols):
            fld = int(f[i] if by_row else f[k])
            X = to_integer(M[:, i, k], fld, s)
            S[:, i, k] = digits(X, s)
    return S, f


def _chunks(V: int, lsb: int, k: int):
    """The k leading 53-bit pieces of |V| (truncated) as signed doubles."""
    if V == 0:
        return [0.0] * k
    neg = V < 0
    a = -V if neg else V
    P = a.bit_length() - 1
    out = []
    for c in range(k):
        sh = P - 52 - 53 * c
        piece = ((a >> sh) if sh >= 0 else (a << -sh)) & ((1 << 53) - 1)
        x = math.ldexp(float(piece), lsb + sh)
        out.append(-x if neg else x)
    return out


def _chunk_dd(V: int, lsb: int):
    hi, lo = _chunks(V, lsb, 2)
    s_ = hi + lo
    bv = s_ - hi
    av = s_ - bv
    return s_, (hi - av) + (lo - bv)


def gemm(A: np.ndarray, B: np.ndarray, s: int = 16, C0=None, mode: str = "set"):
    """DD / QD C (mode) A B by the INT8-slice scheme above; returns (limbs, m, n)."""
    limbs, m, l = A.shape
    n = B.shape[2]
    SA, fa = split(A, s, by_row=True)
    SB, fb = split(B, s, by_row=False)
    D = np.zeros((s + 2, m, n), dtype=np.int64)
    for r in range(2, s + 2):
        for p in range(1, r):
            q = r - p
            D[r] += SA[p - 1] @ SB[q - 1]
    T = 6 + 7 * (s - 1)
    C = np.zeros((limbs, m, n))
    for i in range(m):
        for j in range(n):
            V = 0
            for r in range(2, s + 2):
                V += int(D[r, i, j]) << (7 * (s + 1 - r))
            lsb = (int(fa[i]) - 1022) + (int(fb[j]) - 1022) - T - 6
            if limbs == 2:
                v = np.array(_chunk_dd(V, lsb))
                add = dd_add
            else:
                v = renorm(np.array(_chunks(V, lsb, 4)))
                add = qd_add
            if mode == "add":
                v = add(C0[:, i, j], v)
            elif mode == "sub":
                v = add(C0[:, i, j], -v)
            C[:, i, j] = v
    return C, (SA, SB, D, fa, fb)
