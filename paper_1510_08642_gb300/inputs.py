"""Seeded synthetic operands for DD / QD matrix products.

This module is shared by the tests, the benchmark and the smoke check. It
holds no arithmetic of the method (no products, no TwoSum, no
renormalisation): it only draws random doubles and lays them out as limb
planes, so that the CPU oracle and the CUDA library see identical bits.

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), evaluated as a
counter-based generator: draw i of stream ``seed`` is
``mix(seed * 2**32 + 0x9E3779B97F4A7C15 * (i + 1))``; mix is the published
SplitMix64 finaliser. A draw x becomes u = (x >> 11) * 2**-53 in [0, 1).

Layouts (row-major, leading dimension = number of columns):
  DD matrix: array shape (2, rows, cols): plane 0 = hi, plane 1 = lo.
  QD matrix: array shape (4, rows, cols): limbs x0 (leading) .. x3.

Distributions (the experiment recipes of the paper's Section 3 benchmark and
Section 4 LU tests, and the wide-range case of the INT8-slice product):
  uniform:  hi ~ U[-1, 1) on the 2**-52 grid; every further limb is the
            previous one times 2**-53 * U[-1/2, 1/2), so |x_{k+1}| <
            ulp(x_k) / 2 and the limbs are already normalised.
  wide:     hi = sign * 2**round(N(0, sigma)) with N drawn by Box-Muller
            from two uniforms; further limbs as for uniform.
  integer:  integer-valued hi in [-2**bits, 2**bits], zero lower limbs.
  paper:    the Section 3 test matrices A = [sqrt(5) (i + j - 1)],
            B = [sqrt(3) (n - i)], each entry correctly rounded to DD/QD
            from an integer square root (no floating-point arithmetic).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of SplitMix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        x = np.uint64((seed * (1 << 32)) & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        x = (x ^ (x >> np.uint64(30))) * _M1
        x = (x ^ (x >> np.uint64(27))) * _M2
        x = x ^ (x >> np.uint64(31))
    return x


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """u = (x >> 11) * 2**-53, exactly representable, in [0, 1)."""
    x = splitmix64(seed, count, offset)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _lower_limbs(lead: np.ndarray, limbs: int, seed: int) -> np.ndarray:
    out = np.zeros((limbs,) + lead.shape, dtype=np.float64)
    out[0] = lead
    cnt = lead.size
    for k in range(1, limbs):
        u = uniform01(seed, cnt, offset=k * cnt).reshape(lead.shape) - 0.5
        # scaling by a power of two and by |u| < 1/2 keeps |x_k| < ulp(x_{k-1})/2
        out[k] = out[k - 1] * (2.0 ** -53) * u
    return out


def uniform(rows: int, cols: int, limbs: int = 2, seed: int = 0) -> np.ndarray:
    """DD (limbs=2) or QD (limbs=4) matrix, leading limb ~ U[-1, 1)."""
    cnt = rows * cols
    lead = (2.0 * uniform01(seed, cnt) - 1.0).reshape(rows, cols)
    return _lower_limbs(lead, limbs, seed)


def wide(rows: int, cols: int, limbs: int = 2, seed: int = 0, sigma: float = 8.0) -> np.ndarray:
    """Leading limb sign * 2**round(N(0, sigma)), the wide-range recipe."""
    cnt = rows * cols
    u1 = uniform01(seed, cnt, offset=0)
    u2 = uniform01(seed, cnt, offset=cnt)
    u3 = uniform01(seed, cnt, offset=2 * cnt)
    g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    expo = np.rint(g * sigma)
    sign = np.where(u3 < 0.5, -1.0, 1.0)
    lead = (sign * np.exp2(expo)).reshape(rows, cols)
    # the lower limbs use a seed stream of their own
    return _lower_limbs(lead, limbs, seed + 7919)


def integer(rows: int, cols: int, limbs: int = 2, seed: int = 0, bits: int = 20) -> np.ndarray:
    """Integer-valued leading limb in [-2**bits, 2**bits]; lower limbs zero."""
    cnt = rows * cols
    x = splitmix64(seed, cnt)
    span = np.uint64((1 << (bits + 1)) + 1)
    v = (x % span).astype(np.int64) - (1 << bits)
    out = np.zeros((limbs, rows, cols), dtype=np.float64)
    out[0] = v.reshape(rows, cols).astype(np.float64)
    return out


def _round_sqrt_expansion(k2: int, limbs: int) -> list:
    """sqrt(k2) (k2 a non-negative integer) rounded limb by limb to doubles.

    Each limb is the double nearest to the remaining exact residual, where the
    exact value is known to 400+ bits from math.isqrt; this is plain
    rounding of a real constant, not arithmetic of the method.
    """
    if k2 == 0:
        return [0.0] * limbs
    prec = 480
    root = Fraction(math.isqrt(k2 << (2 * prec)), 1 << prec)
    out = []
    rem = root
    for _ in range(limbs):
        d = _nearest_double(rem)
        out.append(d)
        rem = rem - Fraction(d)
    return out


def _nearest_double(q: Fraction) -> float:
    if q == 0:
        return 0.0
    neg = q < 0
    q = -q if neg else q
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(1 << e if e >= 0 else 1, 1 if e >= 0 else 1 << -e) > q:
        e -= 1
    # q in [2**e, 2**(e+1)); 53-bit significand: scale by 2**(52-e)
    s = q * (Fraction(1 << (52 - e)) if 52 - e >= 0 else Fraction(1, 1 << (e - 52)))
    n = s.numerator // s.denominator
    r = s - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    v = math.ldexp(float(n), e - 52)
    return -v if neg else v


def paper_matrices(n: int, limbs: int = 2) -> tuple:
    """The Section 3 test pair A = [sqrt5 (i+j-1)], B = [sqrt3 (n-i)].

    Entries are indexed from 1 as in the paper. Returns (A, B) with shape
    (limbs, n, n). B depends on the row index only.
    """
    A = np.zeros((limbs, n, n))
    B = np.zeros((limbs, n, n))
    cache = {}
    for s in range(1, 2 * n):
        cache[("a", s)] = _round_sqrt_expansion(5 * s * s, limbs)
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            A[:, i - 1, j - 1] = cache[("a", i + j - 1)]
        B[:, i - 1, :] = np.array(_round_sqrt_expansion(3 * (n - i) ** 2, limbs))[:, None]
    return A, B


def log_uniform_dims(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """count x 3 integer dims, each exp(U[ln lo, ln hi]) rounded."""
    u = uniform01(seed, 3 * count).reshape(count, 3)
    d = np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    return np.clip(d, lo, hi)
