"""The shared input generator: determinism, ranges and normalised limbs."""
import math

import numpy as np

from paper_1510_08642_gb300 import inputs as I


def test_splitmix64_reference_values():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: the published first
    # outputs of the generator with increment 0x9E3779B97F4A7C15.
    x = I.splitmix64(0, 3)
    assert [int(v) for v in x] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_deterministic_and_offsets():
    a = I.uniform01(5, 10)
    b = I.uniform01(5, 4, offset=6)
    assert np.array_equal(a[6:], b)
    assert np.array_equal(I.uniform(7, 9, 2, seed=3), I.uniform(7, 9, 2, seed=3))
    assert not np.array_equal(I.uniform(7, 9, 2, seed=3), I.uniform(7, 9, 2, seed=4))


def _normalised(M):
    for k in range(M.shape[0] - 1):
        hi, lo = M[k], M[k + 1]
        ulp = np.array([math.ulp(v) for v in hi.ravel()]).reshape(hi.shape)
        assert np.all(np.abs(lo) <= ulp / 2)
        assert np.all(hi + lo == hi)


def test_uniform_limbs_normalised():
    for limbs in (2, 4):
        M = I.uniform(33, 17, limbs, seed=1)
        assert np.all(M[0] >= -1) and np.all(M[0] < 1)
        _normalised(M)


def test_wide_range():
    M = I.wide(64, 64, 2, seed=2, sigma=8.0)
    e = np.log2(np.abs(M[0]))
    assert np.all(e == np.round(e))
    assert 5 < np.std(e) < 11
    _normalised(M)


def test_integer_and_dims():
    M = I.integer(10, 10, 2, seed=3, bits=20)
    assert np.all(np.abs(M[0]) <= 2 ** 20) and not M[1].any()
    d = I.log_uniform_dims(1000, 32, 1024, seed=4)
    assert d.min() >= 32 and d.max() <= 1024
    assert 150 < np.exp(np.log(d).mean()) < 250


def test_paper_matrices_rounding():
    A, B = I.paper_matrices(4, 2)
    # A_11 = sqrt(5), B_1j = 3 sqrt(3), B_4j = 0
    assert A[0, 0, 0] == math.sqrt(5.0)
    assert B[0, 0, 0] == math.sqrt(27.0) and B[0, 3, 0] == 0.0
    _normalised(A)
