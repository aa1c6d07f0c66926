"""Pins for the oracle's Simple product (Eq. 1), exact checker and LU.

Each check is fixed by exact arithmetic or by a closed form, never by the
oracle itself:
  * brute-force rational products on tiny dyadic matrices (every limb
    matters, so a dropped cross term, a wrong sign or a transposed operand
    breaks the elementwise bound);
  * integer matrices, where every intermediate fits in 106 bits and the
    result must be exact;
  * identity / permutation / rank-1 / all-ones closed forms;
  * the paper's Section 3 test matrices, whose product has the closed form
    C_ij = sqrt(15) [(i-1) n(n-1)/2 + (n-1) n (n+1)/6];
  * the exact checker against Fraction arithmetic and planted perturbations.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1510_08642_gb300 import inputs as I
from tests.exact import F, U, abs_gemm, exact_gemm, limbs_value, sqrt_fraction

SHAPES = [(1, 1, 1), (3, 5, 2), (4, 4, 4), (5, 2, 7), (2, 7, 3)]


def _val(C, i, j):
    return limbs_value(C[:, i, j])


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("shape", SHAPES)
def test_simple_vs_rational_bruteforce(limbs, shape):
    m, l, n = shape
    A = I.uniform(m, l, limbs, seed=10 + m)
    B = I.uniform(l, n, limbs, seed=20 + n)
    C = O.gemm_simple(A, B)
    ex = exact_gemm(A, B)
    ab = abs_gemm(A, B)
    eps = U * U if limbs == 2 else Fraction(1, 1 << 208)
    # l multiply-adds, each within a few eps of the running magnitudes
    for i in range(m):
        for j in range(n):
            err = abs(_val(C, i, j) - ex[i][j])
            assert err <= 8 * l * eps * ab[i][j], (i, j, float(err), float(ab[i][j]))


@pytest.mark.parametrize("limbs", [2, 4])
def test_simple_detects_lower_limbs(limbs):
    # the lower limbs carry the precision: dropping them would break the bound
    A = I.uniform(4, 6, limbs, seed=3)
    B = I.uniform(6, 5, limbs, seed=4)
    C = O.gemm_simple(A, B)
    ex = exact_gemm(A, B)
    A1 = A.copy()
    A1[1:] = 0
    C1 = O.gemm_simple(A1, B)
    ab = abs_gemm(A, B)
    eps = U * U if limbs == 2 else Fraction(1, 1 << 208)
    bad = max(abs(_val(C1, i, j) - ex[i][j]) / ab[i][j] for i in range(4) for j in range(5))
    good = max(abs(_val(C, i, j) - ex[i][j]) / ab[i][j] for i in range(4) for j in range(5))
    assert good <= 48 * eps < bad


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("mode", ["add", "sub"])
def test_simple_update_modes(limbs, mode):
    A = I.uniform(3, 4, limbs, seed=5)
    B = I.uniform(4, 2, limbs, seed=6)
    C0 = I.uniform(3, 2, limbs, seed=7)
    C = O.gemm_simple(A, B, C0, mode=mode)
    ex = exact_gemm(A, B)
    s = 1 if mode == "add" else -1
    eps = U * U if limbs == 2 else Fraction(1, 1 << 208)
    for i in range(3):
        for j in range(2):
            want = _val(C0, i, j) + s * ex[i][j]
            assert abs(_val(C, i, j) - want) <= 64 * eps


@pytest.mark.parametrize("limbs", [2, 4])
def test_integer_matrices_exact(limbs):
    m, l, n = 9, 64, 7
    A = I.integer(m, l, limbs, seed=1, bits=20)
    B = I.integer(l, n, limbs, seed=2, bits=20)
    C = O.gemm_simple(A, B)
    ex = (A[0].astype(object) @ B[0].astype(object))
    for i in range(m):
        for j in range(n):
            assert _val(C, i, j) == ex[i, j]


@pytest.mark.parametrize("limbs", [2, 4])
def test_identity_permutation_rank1_ones(limbs):
    n = 6
    A = I.uniform(n, n, limbs, seed=8)
    Id = np.zeros((limbs, n, n))
    Id[0] = np.eye(n)
    assert np.array_equal(O.gemm_simple(A, Id), A)
    assert np.array_equal(O.gemm_simple(Id, A), A)
    perm = np.array([3, 0, 5, 1, 4, 2])
    P = np.zeros((limbs, n, n))
    P[0, np.arange(n), perm] = 1.0
    assert np.array_equal(O.gemm_simple(P, A), A[:, perm, :])
    # rank one: A = u 1^T (m x l), B = 1 v^T (l x n) -> c_ij = l u_i v_j
    u = I.integer(5, 1, limbs, seed=9, bits=15)[0, :, 0]
    v = I.integer(1, 4, limbs, seed=10, bits=15)[0, 0, :]
    l = 37
    Au = np.zeros((limbs, 5, l)); Au[0] = u[:, None]
    Bv = np.zeros((limbs, l, 4)); Bv[0] = v[None, :]
    C = O.gemm_simple(Au, Bv)
    assert np.array_equal(C[0], l * np.outer(u, v)) and not C[1:].any()
    ones = np.zeros((limbs, 3, 11)); ones[0] = 1
    onesb = np.zeros((limbs, 11, 2)); onesb[0] = 1
    assert np.array_equal(O.gemm_simple(ones, onesb)[0], np.full((3, 2), 11.0))


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("n", [5, 16])
def test_paper_matrices_closed_form(limbs, n):
    """Section 3 matrices: the product has a closed form in sqrt(15)."""
    A, B = I.paper_matrices(n, limbs)
    C = O.gemm_simple(A, B)
    s15 = sqrt_fraction(15)
    eps = U * U if limbs == 2 else Fraction(1, 1 << 208)
    ab = abs_gemm(A, B)
    for i in range(1, n + 1):
        want = s15 * ((i - 1) * n * (n - 1) // 2 + (n - 1) * n * (n + 1) // 6)
        for j in range(1, n + 1):
            got = _val(C, i - 1, j - 1)
            # input rounding (each input within eps of its real value) plus Eq. 1
            assert abs(got - want) <= (8 * n + 4) * eps * ab[i - 1][j - 1] + Fraction(1, 1 << 400)


@pytest.mark.parametrize("limbs", [2, 4])
def test_exact_checker_vs_rational(limbs):
    m, l, n = 4, 6, 3
    A = I.uniform(m, l, limbs, seed=11)
    B = I.uniform(l, n, limbs, seed=12)
    C = O.gemm_simple(A, B)
    C[0, 1, 1] += 2.0 ** -30  # planted error
    err = O.gemm_error(A, B, C)
    ex = exact_gemm(A, B)
    for i in range(m):
        for j in range(n):
            want = float(ex[i][j] - _val(C, i, j))
            assert err[i, j] == want
    assert abs(err[1, 1] + 2.0 ** -30) < 2.0 ** -80
    # sampled entries agree with the full check
    rows, cols = np.array([0, 3, 1]), np.array([2, 0, 1])
    e2 = O.gemm_error(A, B, C, rows=rows, cols=cols)
    assert np.array_equal(e2, err[rows, cols])


@pytest.mark.parametrize("mode", ["add", "sub"])
def test_exact_checker_update_modes(mode):
    A = I.uniform(3, 5, 2, seed=13)
    B = I.uniform(5, 4, 2, seed=14)
    C0 = I.uniform(3, 4, 2, seed=15)
    C = O.gemm_simple(A, B, C0, mode=mode)
    ex = exact_gemm(A, B)
    err = O.gemm_error(A, B, C, C0=C0, mode=mode)
    s = 1 if mode == "add" else -1
    for i in range(3):
        for j in range(4):
            assert err[i, j] == float(_val(C0, i, j) + s * ex[i][j] - _val(C, i, j))


def test_exact_value_and_dot():
    A = I.uniform(3, 4, 4, seed=16)
    B = I.uniform(4, 2, 4, seed=17)
    ex = exact_gemm(A, B)
    E = O.gemm_exact(A, B)
    for i in range(3):
        for j in range(2):
            assert E[i, j] == float(ex[i][j])
    x = np.array([1e300, 1.0, -1e300, 2.0 ** -1074])
    assert O.exact_dot(x) == 1.0  # sum is 1 + 2^-1074, rounds to 1
    assert O.exact_dot(np.array([3.0, 2.0 ** -600]), np.array([2.0 ** 500, 2.0 ** -400])) == 3.0 * 2.0 ** 500


def test_lu_oracle_solves_section4_system():
    """Section 4 setup: random [-1,1] matrix, x = [0, 1, ..., n-1], b = A x."""
    n = 48
    A = I.uniform(n, n, 2, seed=18)
    X = np.zeros((2, n, 1)); X[0, :, 0] = np.arange(n)
    Bv = O.gemm_simple(A, X)
    LU, ipiv, info = O.dd_getrf(A, pivot=True)
    assert info == 0
    # pivots agree with LAPACK on the leading limbs (no near-ties here)
    import scipy.linalg
    _, piv = scipy.linalg.lu_factor(A[0])
    assert np.array_equal(piv, ipiv)
    # reconstruct P A = L U with the exact checker: residual of L U vs P A
    L = LU.copy(); U_ = LU.copy()
    for k in range(2):
        L[k] = np.tril(LU[k], -1) + (np.eye(n) if k == 0 else 0)
        U_[k] = np.triu(LU[k])
    PA = A.copy()
    for j in range(n):
        p = ipiv[j]
        PA[:, [j, p], :] = PA[:, [p, j], :]
    err = O.gemm_error(L, U_, PA, C0=None)
    # err = exact(L U) - PA  (sign irrelevant): backward error of DD LU
    rel = np.abs(err).max() / (np.abs(A[0]).max())
    assert rel < n * 2.0 ** -100


def test_generic_residual_matches_dd_and_closed_form():
    """orc_residual on DD operands equals the DD checker; on QD operands
    with an exactly representable product, b - A x is exactly 0, and a
    perturbation of one limb of b by 2^-180 shows up exactly."""
    n = 20
    A = I.uniform(n, n, 2, seed=21)
    X = I.uniform(n, 2, 2, seed=22)
    Bv = O.gemm_simple(A, X)
    assert np.array_equal(O.residual(A, X, Bv), O.dd_residual(A, X, Bv))
    Aq = np.zeros((4, n, n)); Aq[0] = np.round(A[0] * 64)
    Xq = np.zeros((4, n, 1)); Xq[0, :, 0] = np.arange(n)
    Bq = np.zeros((4, n, 1)); Bq[0] = Aq[0] @ Xq[0]  # small integers: exact
    assert not np.abs(O.residual(Aq, Xq, Bq)).any()
    Bq[3, 5, 0] = 2.0 ** -180
    r = O.residual(Aq, Xq, Bq)
    assert r[5, 0] == 2.0 ** -180 and np.count_nonzero(r) == 1


def test_qd_lu_oracle_reconstructs_PA():
    """Unblocked QD LU: pivots as LAPACK on the leading limbs, and
    L U = P A to QD accuracy (exact checker on the QD product)."""
    n = 40
    A = I.uniform(n, n, 4, seed=23)
    LU, ipiv, info = O.qd_getrf(A, pivot=True)
    assert info == 0
    import scipy.linalg
    _, piv = scipy.linalg.lu_factor(A[0])
    assert np.array_equal(piv, ipiv)
    L = np.zeros_like(LU); U_ = np.zeros_like(LU)
    for k in range(4):
        L[k] = np.tril(LU[k], -1) + (np.eye(n) if k == 0 else 0)
        U_[k] = np.triu(LU[k])
    PA = A.copy()
    for j in range(n):
        p = ipiv[j]
        PA[:, [j, p], :] = PA[:, [p, j], :]
    err = O.gemm_error(L, U_, PA, C0=None)
    assert np.abs(err).max() / np.abs(A[0]).max() < n * 2.0 ** -200
    # a zero column is reported as 1 + its index
    A[:, :, 9] = 0.0
    assert O.qd_getrf(A, pivot=True)[2] == 10


def test_qd_lu_solution_of_section4_system():
    """QD LU + substitution in the oracle (plain QD sums on the factors):
    residual of the Section 4 system below n 2^-200."""
    n = 24
    A = I.uniform(n, n, 4, seed=24)
    X = np.zeros((4, n, 1)); X[0, :, 0] = np.arange(n)
    Bv = O.gemm_simple(A, X)
    LU, ipiv, info = O.qd_getrf(A)
    y = [np.array(Bv[:, i, 0]) for i in range(n)]
    for j in range(n):
        y[j], y[ipiv[j]] = y[ipiv[j]], y[j]
    for i in range(n):
        for k in range(i):
            y[i] = O.qd_add(y[i], O.qd_mul(-LU[:, i, k], y[k]))
    for i in reversed(range(n)):
        for k in range(i + 1, n):
            y[i] = O.qd_add(y[i], O.qd_mul(-LU[:, i, k], y[k]))
        y[i] = O.qd_div(y[i], LU[:, i, i])
    Xh = np.stack(y, axis=1)[:, :, None]
    r = O.residual(A, Xh, Bv)
    assert np.abs(r).max() / (np.abs(A[0]).sum(axis=1).max() * np.abs(Xh[0]).max()) <= n * 2.0 ** -200
