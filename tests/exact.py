"""Exact rational helpers for the tests (independent of the oracle's C++)."""
from fractions import Fraction
import math

import numpy as np

U = Fraction(1, 1 << 53)  # unit roundoff of binary64


def F(x) -> Fraction:
    return Fraction(float(x))


def limbs_value(v) -> Fraction:
    return sum((F(x) for x in v), Fraction(0))


def ulp(x: float) -> float:
    x = abs(float(x))
    if x == 0.0:
        return 2.0 ** -1074
    return math.ulp(x)


def exact_gemm(A: np.ndarray, B: np.ndarray):
    """Exact product of limb-plane matrices as a nested list of Fractions."""
    limbs, m, l = A.shape
    n = B.shape[2]
    a = [[limbs_value(A[:, i, k]) for k in range(l)] for i in range(m)]
    b = [[limbs_value(B[:, k, j]) for j in range(n)] for k in range(l)]
    return [[sum((a[i][k] * b[k][j] for k in range(l)), Fraction(0)) for j in range(n)]
            for i in range(m)]


def abs_gemm(A: np.ndarray, B: np.ndarray):
    """sum_k |a_ik| |b_kj| (exact) for elementwise bounds."""
    limbs, m, l = A.shape
    n = B.shape[2]
    a = [[abs(limbs_value(A[:, i, k])) for k in range(l)] for i in range(m)]
    b = [[abs(limbs_value(B[:, k, j])) for j in range(n)] for k in range(l)]
    return [[sum((a[i][k] * b[k][j] for k in range(l)), Fraction(0)) for j in range(n)]
            for i in range(m)]


def sqrt_fraction(k2: int, bits: int = 480) -> Fraction:
    """floor(sqrt(k2) * 2**bits) / 2**bits: within 2**-bits of sqrt(k2)."""
    return Fraction(math.isqrt(k2 << (2 * bits)), 1 << bits)
