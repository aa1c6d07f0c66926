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

The CRT variant (Ozaki, Uchino, Imamura 2025, "scheme II"; DDG_OZAKI2):
1. moduli m_1 > m_2 > ... > m_N: the N largest pairwise-coprime integers
   <= 256, taken greedily from 256 downward; M = m_1 ... m_N;
2. P = min(120, floor((bitlen(M) - 2 - ceil(log2 l)) / 2)), so that
   l 2^(2P) < M / 2;
3. X_ik = round-half-up of a_ik 2^(P - e_i) (step 2 above with T = P),
   likewise Y_kj per column;
4. Z = X Y exactly. The library obtains Z from the residues Z mod m_t (one
   INT8 product per modulus) by the Chinese remainder theorem, which is exact
   because |Z| <= l 2^(2P) < M / 2; the oracle forms Z directly;
5. c = Z 2^(e_i + e_j - 2P) rounded to DD as in step 5.
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
    return to_integer_T(limbs, field, 6 + 7 * (s - 1))


def to_integer_T(limbs, field: int, T: int) -> int:
    """round-half-up of x 2^(T - e), e = field - 1022, each limb truncated
    toward zero at 2^-64 units first."""
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


# ------------------------------------------------------------- CRT scheme --
def crt_moduli(N: int) -> list:
    """The N largest pairwise-coprime integers <= 256, greedily from 256 down."""
    out = []
    m = 256
    while len(out) < N and m > 1:
        if all(math.gcd(m, x) == 1 for x in out):
            out.append(m)
        m -= 1
    if len(out) < N:
        raise ValueError("not enough moduli")
    return out


def crt_precision(N: int, l: int) -> int:
    """Bits P of the integer scaling: l 2^(2P) < M / 2, at most 120."""
    M = math.prod(crt_moduli(N))
    clog = (max(l, 1) - 1).bit_length()
    return min(120, (M.bit_length() - 2 - clog) // 2)


def crt_reconstruct(residues, moduli) -> int:
    """The integer Z with |Z| < M / 2 and Z = r_t (mod m_t) for every t."""
    M = math.prod(moduli)
    z = 0
    for r, m in zip(residues, moduli):
        Mt = M // m
        z += r * Mt * pow(Mt, -1, m)
    z %= M
    return z - M if 2 * z >= M else z


def gemm_crt(A: np.ndarray, B: np.ndarray, N: int = 32, C0=None, mode: str = "set"):
    """DD C (mode) A B by the CRT scheme above; returns (2, m, n)."""
    limbs, m, l = A.shape
    assert limbs == 2
    n = B.shape[2]
    P = crt_precision(N, l)
    if P < 1:
        raise ValueError("too few moduli for this l")
    fa = row_fields(A[0], axis=1)
    fb = row_fields(B[0], axis=0)
    X = np.empty((m, l), dtype=object)
    Y = np.empty((l, n), dtype=object)
    for i in range(m):
        for k in range(l):
            X[i, k] = to_integer_T(A[:, i, k], int(fa[i]), P)
    for k in range(l):
        for j in range(n):
            Y[k, j] = to_integer_T(B[:, k, j], int(fb[j]), P)
    Z = X.dot(Y) if l else np.zeros((m, n), dtype=object)
    C = np.zeros((2, m, n))
    for i in range(m):
        for j in range(n):
            lsb = (int(fa[i]) - 1022) + (int(fb[j]) - 1022) - 2 * P
            v = np.array(_chunk_dd(int(Z[i, j]), lsb))
            if mode == "add":
                v = dd_add(C0[:, i, j], v)
            elif mode == "sub":
                v = dd_add(C0[:, i, j], -v)
            C[:, i, j] = v
    return C, (X, Y, Z, fa, fb, P)


def gemm_crt_entries(A: np.ndarray, B: np.ndarray, N: int, rows, cols) -> np.ndarray:
    """Entries (rows[t], cols[t]) of gemm_crt(A, B, N), one by one: (2, count)."""
    limbs, m, l = A.shape
    P = crt_precision(N, l)
    out = np.zeros((2, len(rows)))
    for t, (i, j) in enumerate(zip(rows, cols)):
        fa = int(row_fields(A[0][i:i + 1], axis=1)[0])
        fb = int(row_fields(B[0][:, j:j + 1], axis=0)[0])
        Z = 0
        for k in range(l):
            Z += to_integer_T(A[:, i, k], fa, P) * to_integer_T(B[:, k, j], fb, P)
        out[:, t] = _chunk_dd(Z, (fa - 1022) + (fb - 1022) - 2 * P)
    return out
