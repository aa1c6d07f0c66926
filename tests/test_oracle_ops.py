"""Pins for the oracle's scalar DD / QD operations.

Every check compares against exact rational arithmetic (fractions.Fraction),
never against the oracle itself: error-free transformations must be exact,
and the DD / QD operations must meet their published error bounds
(Joldes, Muller, Popescu 2017 for the double-word sum and product; a few
units of 2**-212 for the four-limb operations) and keep their limbs
normalised.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests.exact import F, U, limbs_value, ulp

pytestmark = pytest.mark.filterwarnings("ignore")


def rand_double(rng, lo=-60, hi=60):
    return rng.choice([-1.0, 1.0]) * math.ldexp(rng.random() + 0.5, rng.randint(lo, hi))


def rand_dd(rng, e=0):
    hi = rand_double(rng, e, e)
    lo = hi * 2.0 ** -53 * (rng.random() - 0.5)
    return np.array([hi, lo])


def rand_qd(rng, e=0):
    x = [rand_double(rng, e, e)]
    for _ in range(3):
        x.append(x[-1] * 2.0 ** -53 * (rng.random() - 0.5))
    return np.array(x)


EDGE = [0.0, 1.0, -1.0, 0.5, 2.0 ** 52, 2.0 ** -52, 1.0 + 2.0 ** -52, 3.0, 1e300, 1e-300,
        -(2.0 ** 60) + 1.0, 0.1, -0.7, 2.0 ** 1000, 2.0 ** -1000]


def test_two_sum_exact():
    rng = random.Random(1)
    pairs = [(a, b) for a in EDGE for b in EDGE if abs(a) < 1e300 and abs(b) < 1e300]
    pairs += [(rand_double(rng), rand_double(rng)) for _ in range(3000)]
    for a, b in pairs:
        s, e = O.two_sum(a, b)
        assert s == a + b
        assert F(s) + F(e) == F(a) + F(b)


def test_two_prod_exact():
    rng = random.Random(2)
    pairs = [(rand_double(rng, -400, 400), rand_double(rng, -400, 400)) for _ in range(3000)]
    pairs += [(a, b) for a in EDGE for b in EDGE if 1e-250 < abs(a * b) < 1e250]
    for a, b in pairs:
        p, e = O.two_prod(a, b)
        assert p == a * b
        assert F(p) + F(e) == F(a) * F(b)


def dd_normalised(r):
    return r[0] + r[1] == r[0] and abs(r[1]) <= ulp(r[0]) / 2


def test_dd_mul_bound_and_normalisation():
    rng = random.Random(3)
    worst = Fraction(0)
    for t in range(4000):
        a, b = rand_dd(rng, rng.randint(-30, 30)), rand_dd(rng, rng.randint(-30, 30))
        if t % 7 == 0:
            b = np.array([1.0, 0.0])
        r = O.dd_mul(a, b)
        ex = limbs_value(a) * limbs_value(b)
        err = abs(limbs_value(r) - ex)
        assert dd_normalised(r)
        if ex != 0:
            worst = max(worst, err / abs(ex))
    # dropped lo*lo (<= u^2), two rounded FMAs on the error term (<= 2u^2 each)
    assert worst <= 5 * U * U
    assert worst > 0  # the operation is not exact in general


def test_dd_mul_by_one_and_zero_exact():
    rng = random.Random(4)
    for _ in range(200):
        a = rand_dd(rng)
        assert np.array_equal(O.dd_mul(a, [1.0, 0.0]), a)
        assert limbs_value(O.dd_mul(a, [0.0, 0.0])) == 0


def test_dd_add_bound_including_cancellation():
    rng = random.Random(5)
    worst = Fraction(0)
    for t in range(4000):
        a = rand_dd(rng, rng.randint(-5, 5))
        if t % 3 == 0:  # heavy cancellation
            b = np.array([-a[0], a[1] * (rng.random() - 0.5)])
        elif t % 3 == 1:
            b = np.array([-a[0] * (1 + 2.0 ** -50), rand_double(rng, -80, -60)])
        else:
            b = rand_dd(rng, rng.randint(-5, 5))
        r = O.dd_add(a, b)
        ex = limbs_value(a) + limbs_value(b)
        err = abs(limbs_value(r) - ex)
        assert dd_normalised(r)
        if ex != 0:
            worst = max(worst, err / abs(ex))
        else:
            assert err == 0
    assert worst <= 3 * U * U * (1 + 8 * U)  # accurate double-word sum bound


def qd_separated(r):
    """Limbs strictly decreasing: |x_{k+1}| <= 2**-40 |x_k| (zeros trail).

    The renormalisation emits a limb as soon as a TwoSum leaves an error, so
    a later limb may exceed ulp(x_k) by a small factor when the terms of the
    product arrive in near-equal pairs; the limbs stay 40+ bits apart and
    the accuracy bound below is what callers rely on.
    """
    for k in range(3):
        if r[k] == 0:
            return all(x == 0 for x in r[k + 1:])
        if not abs(r[k + 1]) <= abs(r[k]) * 2.0 ** -40:
            return False
    return True


def test_qd_mul_bound():
    rng = random.Random(6)
    worst = Fraction(0)
    for _ in range(2000):
        a, b = rand_qd(rng, rng.randint(-20, 20)), rand_qd(rng, rng.randint(-20, 20))
        r = O.qd_mul(a, b)
        ex = limbs_value(a) * limbs_value(b)
        rel = abs(limbs_value(r) - ex) / abs(ex)
        worst = max(worst, rel)
        assert qd_separated(r)
    assert worst <= Fraction(1, 1 << 210)
    assert worst > 0


def test_qd_add_bound_including_cancellation():
    rng = random.Random(7)
    worst = Fraction(0)
    for t in range(2000):
        a = rand_qd(rng, rng.randint(-3, 3))
        if t % 2 == 0:
            b = np.array([-a[0], -a[1], rand_double(rng, -170, -160), 0.0])
        else:
            b = rand_qd(rng, rng.randint(-40, 3))
        r = O.qd_add(a, b)
        ex = limbs_value(a) + limbs_value(b)
        assert qd_separated(r)
        if ex == 0:
            assert limbs_value(r) == 0
            continue
        worst = max(worst, abs(limbs_value(r) - ex) / abs(ex))
    assert worst <= Fraction(1, 1 << 208)


def test_qd_add_exact_cases():
    rng = random.Random(8)
    for _ in range(200):
        a = rand_qd(rng)
        assert limbs_value(O.qd_add(a, -a)) == 0
        z = O.qd_add(a, np.zeros(4))
        assert limbs_value(z) == limbs_value(a)


def test_renorm_reproduces_short_sums_exactly():
    rng = random.Random(9)
    for _ in range(500):
        # terms spread over fewer than 4 * 53 bits sum exactly into 4 limbs
        x = [rand_double(rng, -5, 5) for _ in range(3)]
        r = O.renorm(np.array(x))
        assert limbs_value(r) == sum(F(v) for v in x)


def test_qd_div_bound():
    """QD long division (the LU quotients): |a/b - q| <= 2^-205 |a/b|."""
    rng = random.Random(9)
    worst = Fraction(0)
    for _ in range(1000):
        a, b = rand_qd(rng, rng.randint(-20, 20)), rand_qd(rng, rng.randint(-20, 20))
        q = O.qd_div(a, b)
        ex = limbs_value(a) / limbs_value(b)
        worst = max(worst, abs(limbs_value(q) - ex) / abs(ex))
        assert qd_separated(q)
    assert 0 < worst <= Fraction(1, 1 << 205)
    # exact quotients stay exact
    assert np.array_equal(O.qd_div([6.0, 0, 0, 0], [3.0, 0, 0, 0]), [2.0, 0, 0, 0])
    assert np.array_equal(O.qd_div([0.0, 0, 0, 0], [3.0, 0, 0, 0]), [0.0, 0, 0, 0])


def sparse_qd(rng):
    """QD numbers whose lower limbs sit far below their positions (an
    integer or short value plus tiny corrections, as in LU solutions)."""
    x = [rand_double(rng, -3, 3)]
    if rng.random() < 0.3:
        x[0] = float(rng.randint(1, 1000)) * rng.choice([-1.0, 1.0])
    for _ in range(3):
        gap = rng.choice([53, 54, 60, 80, 106, 150, 300])
        x.append(x[-1] * 2.0 ** -gap * (rng.random() - 0.5) if rng.random() < 0.9 else 0.0)
    return O.renorm(np.array(x))


def test_qd_mul_bound_sparse_limbs():
    """The QD product keeps the 2^-210 bound when limbs are far below their
    positions (without ordering its terms by magnitude the renormalisation
    spends limbs on overlapping pieces: ~2^-160 on these inputs)."""
    rng = random.Random(10)
    worst = Fraction(0)
    for _ in range(1500):
        a, b = sparse_qd(rng), sparse_qd(rng)
        r = O.qd_mul(a, b)
        ex = limbs_value(a) * limbs_value(b)
        if ex:
            worst = max(worst, abs(limbs_value(r) - ex) / abs(ex))
        assert qd_separated(r)
    # the failing case of an LU back substitution: x = 23 + 2^-208-ish
    a = np.array([-3.70949070e+00, 1.68262898e-18, -1.75943975e-35, -2.09907835e-52])
    b = np.array([2.3e+01, -5.24109001e-63, 1.02562329e-79, -5.68207668e-96])
    a, b = O.renorm(a), O.renorm(b)
    r = O.qd_mul(a, b)
    ex = limbs_value(a) * limbs_value(b)
    worst = max(worst, abs(limbs_value(r) - ex) / abs(ex))
    assert worst <= Fraction(1, 1 << 210)
