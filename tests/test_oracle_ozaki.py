"""Pins for the INT8-slice oracle (oracle/ozaki.py), against exact arithmetic.

* the integer X is within 1/2 + 2^-63 of a 2^(T - e) (rounding);
* the balanced digits reconstruct X exactly and lie in [-64, 64];
* every product of digit slices is exact in INT32 for the sizes used;
* the whole result is within its error bound of the exact product
  (Kulisch checker) and exact for integer matrices with enough slices.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import oracle.ozaki as OZ
from paper_1510_08642_gb300 import inputs as I


@pytest.mark.parametrize("s", [4, 9, 16])
def test_split_reconstructs(s):
    A = I.uniform(5, 9, 2, seed=1)
    A[:, 2, 3] = 0.0
    A[:, 4, :] *= 2.0 ** -40
    T = 6 + 7 * (s - 1)
    S, f = OZ.split(A, s, by_row=True)
    assert np.all(np.abs(S) <= 64)
    assert np.all(np.abs(S[1:]) <= 64) and np.all(S[1:] >= -64) and np.all(S[1:] <= 63)
    for i in range(5):
        e = int(f[i]) - 1022
        for k in range(9):
            X = sum(int(S[p, i, k]) * 128 ** (s - 1 - p) for p in range(s))
            exact = (Fraction(float(A[0, i, k])) + Fraction(float(A[1, i, k]))) * Fraction(2) ** (T - e)
            assert abs(X - exact) <= Fraction(1, 2) + Fraction(1, 1 << 62)
            assert abs(exact) < Fraction(2) ** T


def test_digits_balanced_cases():
    s = 5
    for X in [0, 1, -1, 63, 64, -64, 127, 128, -129, 64 * 128 ** 4, -64 * 128 ** 4, 12345678, -987654321]:
        d = OZ.digits(X, s)
        assert sum(v * 128 ** (s - 1 - p) for p, v in enumerate(d)) == X
        assert all(-64 <= v <= 63 for v in d[1:])


@pytest.mark.parametrize("s", [8, 12, 16])
def test_ozaki_within_bound(s):
    m, l, n = 7, 33, 6
    A = I.uniform(m, l, 2, seed=2)
    B = I.uniform(l, n, 2, seed=3)
    C, (SA, SB, D, fa, fb) = OZ.gemm(A, B, s)
    assert np.abs(D).max() < 2 ** 31
    err = O.gemm_error(A, B, C)
    for i in range(m):
        for j in range(n):
            scale = 2.0 ** (int(fa[i]) - 1022 + int(fb[j]) - 1022)
            assert abs(err[i, j]) <= l * (s + 3) * 2.0 ** (-7 * s) * scale + 2.0 ** -104 * scale


def test_ozaki_integer_exact():
    A = I.integer(6, 20, 2, seed=4, bits=20)
    B = I.integer(20, 5, 2, seed=5, bits=20)
    C, _ = OZ.gemm(A, B, 8)
    assert not O.gemm_error(A, B, C).any()


def test_ozaki_modes():
    A = I.uniform(4, 10, 2, seed=6)
    B = I.uniform(10, 3, 2, seed=7)
    C0 = I.uniform(4, 3, 2, seed=8)
    for mode in ("add", "sub"):
        C, _ = OZ.gemm(A, B, 16, C0=C0, mode=mode)
        err = O.gemm_error(A, B, C, C0=C0, mode=mode)
        assert np.abs(err).max() < 2.0 ** -95


@pytest.mark.parametrize("s", [12, 24, 32])
def test_ozaki_qd_within_bound(s):
    m, l, n = 5, 21, 4
    A = I.uniform(m, l, 4, seed=20)
    B = I.uniform(l, n, 4, seed=21)
    C, (SA, SB, D, fa, fb) = OZ.gemm(A, B, s)
    assert np.abs(D).max() < 2 ** 31
    err = O.gemm_error(A, B, C)
    for i in range(m):
        for j in range(n):
            scale = 2.0 ** (int(fa[i]) - 1022 + int(fb[j]) - 1022)
            assert abs(err[i, j]) <= l * (s + 3) * 2.0 ** (-7 * s) * scale + 2.0 ** -208 * scale


def test_ozaki_qd_split_reconstructs():
    s = 32
    A = I.uniform(3, 5, 4, seed=22)
    T = 6 + 7 * (s - 1)
    S, f = OZ.split(A, s, by_row=True)
    assert np.all(np.abs(S) <= 64)
    for i in range(3):
        e = int(f[i]) - 1022
        for k in range(5):
            X = sum(int(S[p, i, k]) * 128 ** (s - 1 - p) for p in range(s))
            exact = sum(Fraction(float(A[q, i, k])) for q in range(4)) * Fraction(2) ** (T - e)
            assert abs(X - exact) <= Fraction(1, 2) + Fraction(4, 1 << 64)


# ------------------------------------------------ CRT scheme (DDG_OZAKI2) --
def test_crt_moduli_pairwise_coprime_and_greedy():
    import math
    ms = OZ.crt_moduli(40)
    assert ms[:8] == [256, 255, 253, 251, 247, 241, 239, 233]  # worked by hand
    assert all(2 <= m <= 256 for m in ms) and ms == sorted(ms, reverse=True)
    for a in range(len(ms)):
        for b in range(a):
            assert math.gcd(ms[a], ms[b]) == 1
    # greedy: every skipped integer shares a factor with a larger chosen one
    for x in range(ms[-1] + 1, 257):
        if x not in ms:
            assert any(math.gcd(x, m) > 1 for m in ms if m > x)


@pytest.mark.parametrize("l", [1, 2, 3, 33, 4096, 4097, 65536])
def test_crt_precision_keeps_Z_below_half_M(l):
    import math
    for N in range(2, 41):
        P = OZ.crt_precision(N, l)
        M = math.prod(OZ.crt_moduli(N))
        assert P <= 120
        if P >= 1:
            assert 2 * l * 4 ** P < M


def test_crt_reconstruct_exact_including_extremes():
    import math
    import random
    rng = random.Random(5)
    for N in (2, 7, 32, 40):
        ms = OZ.crt_moduli(N)
        M = math.prod(ms)
        cases = [0, 1, -1, (M - 1) // 2, -((M - 1) // 2)] + [rng.randrange(-(M // 2) + 1, M // 2) for _ in range(50)]
        for z in cases:
            assert OZ.crt_reconstruct([z % m for m in ms], ms) == z


def test_crt_residue_products_give_Z():
    """Step 4 as the library runs it: one int64 product of the residue
    matrices per modulus, reduced, then the CRT, equals X Y exactly."""
    A = I.uniform(5, 17, 2, seed=30)
    B = I.uniform(17, 4, 2, seed=31)
    N = 32
    C, (X, Y, Z, fa, fb, P) = OZ.gemm_crt(A, B, N)
    ms = OZ.crt_moduli(N)
    R = []
    for m in ms:
        Xm = np.vectorize(lambda v: ((v % m) + 128) % m - 128 if m > 128 else v % m, otypes=[np.int64])(X)
        Ym = np.vectorize(lambda v: ((v % m) + 128) % m - 128 if m > 128 else v % m, otypes=[np.int64])(Y)
        assert np.abs(Xm).max() <= 128 and np.abs(Ym).max() <= 128
        R.append((Xm @ Ym) % m)
    for i in range(5):
        for j in range(4):
            assert OZ.crt_reconstruct([int(r[i, j]) for r in R], ms) == Z[i, j]


@pytest.mark.parametrize("N", [20, 26, 32])
def test_crt_within_bound(N):
    """|c - ab| <= l 2^-P 2^(e_i + e_j) (integer rounding of both operands)
    + 2^-104 |c| (the final rounding to DD)."""
    m, l, n = 6, 33, 5
    A = I.uniform(m, l, 2, seed=32)
    B = I.uniform(l, n, 2, seed=33)
    C, (X, Y, Z, fa, fb, P) = OZ.gemm_crt(A, B, N)
    assert P == OZ.crt_precision(N, l)
    err = O.gemm_error(A, B, C)
    worst = 0.0
    for i in range(m):
        for j in range(n):
            scale = 2.0 ** (int(fa[i]) - 1022 + int(fb[j]) - 1022)
            bound = l * 2.0 ** -P * (1 + 2.0 ** -40) * scale + 2.0 ** -104 * abs(C[0, i, j])
            assert abs(err[i, j]) <= bound
            worst = max(worst, abs(err[i, j]) / bound)
    assert worst > 2.0 ** -30  # the bound is not vacuous


def test_crt_integer_exact_and_modes():
    A = I.integer(6, 20, 2, seed=34, bits=20)
    B = I.integer(20, 5, 2, seed=35, bits=20)
    C, _ = OZ.gemm_crt(A, B, 32)
    assert not O.gemm_error(A, B, C).any()
    A = I.uniform(4, 10, 2, seed=36)
    B = I.uniform(10, 3, 2, seed=37)
    C0 = I.uniform(4, 3, 2, seed=38)
    for mode in ("add", "sub"):
        C, _ = OZ.gemm_crt(A, B, 32, C0=C0, mode=mode)
        err = O.gemm_error(A, B, C, C0=C0, mode=mode)
        assert np.abs(err).max() < 2.0 ** -95
