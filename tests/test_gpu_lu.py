"""GPU parity for the Section 4 LU: dd_getrf / dd_getrs through the C ABI.

* Residuals b - A x^ are computed exactly by the oracle (Kulisch
  accumulator): ||b - A x^||_inf / (||A||_inf ||x^||_inf) <= n 2^-100.
* With partial pivoting the pivot sequence equals the oracle's unblocked LU
  (same DD comparison rule) on random matrices.
* Without pivoting (the paper's setting) the factors agree with the oracle's
  unblocked LU to DD accuracy on a diagonally dominant matrix.
* The paper's test problem: random entries in [-1, 1], true solution
  x = [0, 1, ..., n-1], b = A x; Winograd and Block trailing updates give
  errors of the same size (Section 4: no visible loss from Winograd).
* A zero pivot is reported (DDG_ESINGULAR, or through the info word).
"""
import numpy as np
import pytest

import oracle as O
from paper_1510_08642_gb300 import inputs as I
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def section4_problem(n, seed, nrhs=1):
    A = I.uniform(n, n, 2, seed=seed)
    X = np.zeros((2, n, nrhs))
    for c in range(nrhs):
        X[0, :, c] = np.arange(n) + c
    Bv = O.gemm_simple(A, X)
    return A, X, Bv


def lu_solve(A, Bv, K, pivot=True, algo="winograd", cutoff=16):
    import paper_1510_08642_gb300 as P
    dA = to_dev(A)
    ipiv = P.getrf(dA, K=K, pivot=pivot, algo=algo, cutoff=cutoff)
    dB = to_dev(Bv)
    P.getrs(dA, ipiv, dB)
    torch.cuda.synchronize()
    return to_host(dA), ipiv.cpu().numpy(), to_host(dB)


def rel_residual(A, Xh, Bv):
    r = O.dd_residual(A, Xh, Bv)
    if not np.abs(r).max():
        return 0.0
    return np.abs(r).max() / (np.abs(A[0]).sum(axis=1).max() * np.abs(Xh[0]).max())


@pytest.mark.parametrize("n,K,cutoff", [(1, 1, 8), (7, 3, 2), (100, 16, 8), (257, 64, 16), (300, 1, 8),
                                        (129, 512, 16)])
def test_getrf_getrs_residual_and_pivots(n, K, cutoff):
    A, X, Bv = section4_problem(n, seed=n)
    LU, ipiv, Xh = lu_solve(A, Bv, K, cutoff=cutoff)
    assert rel_residual(A, Xh, Bv) <= n * 2.0 ** -100
    _, piv_o, info = O.dd_getrf(A, pivot=True)
    assert info == 0
    assert np.array_equal(ipiv, piv_o)


def test_multiple_rhs():
    n = 150
    A, X, Bv = section4_problem(n, seed=3, nrhs=5)
    _, _, Xh = lu_solve(A, Bv, K=32)
    assert rel_residual(A, Xh, Bv) <= n * 2.0 ** -100


def test_no_pivot_matches_oracle_factors():
    n = 96
    A = I.uniform(n, n, 2, seed=4)
    A[0] += np.eye(n) * n  # diagonally dominant: no pivoting needed
    import paper_1510_08642_gb300 as P
    dA = to_dev(A)
    ipiv = P.getrf(dA, K=32, pivot=False, algo="winograd", cutoff=8)
    torch.cuda.synchronize()
    LU = to_host(dA)
    LUo, piv_o, info = O.dd_getrf(A, pivot=False)
    assert info == 0 and np.array_equal(ipiv.cpu().numpy(), np.arange(n))
    diff = np.abs((LU[0] - LUo[0]) + (LU[1] - LUo[1]))
    assert diff.max() <= 2.0 ** -96 * max(1.0, np.abs(LUo[0]).max())


def test_zero_pivot_reported():
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    n = 40
    A = I.uniform(n, n, 2, seed=5)
    A[:, :, 7] = 0.0  # singular: column 7 is zero
    dA = to_dev(A)
    with pytest.raises(capi.DDGError) as e:
        P.getrf(dA, K=16)
    assert e.value.status == capi.DDG_ESINGULAR
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    dA = to_dev(A)
    P.getrf(dA, K=16, info=info)
    torch.cuda.synchronize()
    assert int(info.item()) == 8


@pytest.mark.parametrize("n", [1024])
def test_section4_winograd_vs_block(n):
    """alpha = 2, n_min = 32 (K = 64): the paper's best DD setting."""
    A, X, Bv = section4_problem(n, seed=11)
    errs = {}
    for algo in ("winograd", "block"):
        _, _, Xh = lu_solve(A, Bv, K=64, algo=algo, cutoff=32)
        assert rel_residual(A, Xh, Bv) <= n * 2.0 ** -100
        fe = np.abs((Xh[0] - X[0]) + Xh[1]) / np.maximum(np.abs(X[0]), 1)
        errs[algo] = fe.max()
    # cond ~ 1e6..1e7 (Section 4): forward error ~ cond * 2^-104, both similar
    assert errs["winograd"] < 1e-20 and errs["block"] < 1e-20
    assert errs["winograd"] < 100 * errs["block"] + 1e-28


# ------------------------------------------------------------------ QD LU --
def qd_problem(n, seed, nrhs=1):
    A = I.uniform(n, n, 4, seed=seed)
    X = np.zeros((4, n, nrhs))
    for c in range(nrhs):
        X[0, :, c] = np.arange(n) + c
    return A, X, O.gemm_simple(A, X)


def qd_rel_residual(A, Xh, Bv):
    r = O.residual(A, Xh, Bv)
    if not np.abs(r).max():
        return 0.0
    return np.abs(r).max() / (np.abs(A[0]).sum(axis=1).max() * np.abs(Xh[0]).max())


@pytest.mark.parametrize("n,K,cutoff,algo", [(1, 1, 8, "winograd"), (9, 4, 2, "winograd"),
                                             (100, 16, 8, "winograd"), (161, 64, 16, "strassen"),
                                             (130, 1, 8, "block"), (97, 512, 16, "winograd")])
def test_qd_getrf_getrs_residual_and_pivots(n, K, cutoff, algo):
    """qd_getrf / qd_getrs: exact residual <= n 2^-200 (QD unit 2^-212 with
    the growth of a pivoted LU), pivots equal to the oracle's unblocked QD LU."""
    A, X, Bv = qd_problem(n, seed=100 + n)
    LU, ipiv, Xh = lu_solve(A, Bv, K, cutoff=cutoff, algo=algo)
    assert qd_rel_residual(A, Xh, Bv) <= n * 2.0 ** -200
    _, piv_o, info = O.qd_getrf(A, pivot=True)
    assert info == 0
    assert np.array_equal(ipiv, piv_o)


def test_qd_no_pivot_matches_oracle_factors():
    n = 72
    A = I.uniform(n, n, 4, seed=41)
    A[0] += np.eye(n) * n
    import paper_1510_08642_gb300 as P
    dA = to_dev(A)
    ipiv = P.getrf(dA, K=16, pivot=False, algo="winograd", cutoff=8)
    torch.cuda.synchronize()
    LU = to_host(dA)
    LUo, _, info = O.qd_getrf(A, pivot=False)
    assert info == 0 and np.array_equal(ipiv.cpu().numpy(), np.arange(n))
    from fractions import Fraction
    worst = 0.0
    for i in range(0, n, 7):
        for j in range(0, n, 5):
            d = sum(Fraction(float(v)) for v in LU[:, i, j]) - sum(Fraction(float(v)) for v in LUo[:, i, j])
            worst = max(worst, abs(float(d)))
    assert worst <= 2.0 ** -196 * max(1.0, np.abs(LUo[0]).max())


def test_qd_zero_pivot_reported():
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    n = 33
    A = I.uniform(n, n, 4, seed=42)
    A[:, :, 20] = 0.0
    with pytest.raises(capi.DDGError) as e:
        P.getrf(to_dev(A), K=8)
    assert e.value.status == capi.DDG_ESINGULAR
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    P.getrf(to_dev(A), K=8, info=info)
    torch.cuda.synchronize()
    assert int(info.item()) == 21


def test_qd_section4_forward_error():
    """The paper's QD setting (Winograd trailing updates): forward error of
    x = [0, 1, ..., n-1] at cond * 2^-212 level, far below DD's."""
    n = 384
    A, X, Bv = qd_problem(n, seed=43)
    _, _, Xh = lu_solve(A, Bv, K=64, algo="winograd", cutoff=32)
    assert qd_rel_residual(A, Xh, Bv) <= n * 2.0 ** -200
    from fractions import Fraction
    fe = max(abs(float(sum(Fraction(float(v)) for v in Xh[:, i, 0]) - i)) / max(i, 1) for i in range(n))
    assert fe < 1e-50


@pytest.mark.parametrize("algo", ["ozaki", "ozaki2"])
def test_int8_trailing_updates(algo):
    """DD LU whose trailing updates are INT8 products (slices / residues +
    CRT): normwise-accurate updates keep the exact residual below n 2^-100
    and the pivots of the oracle's unblocked LU."""
    n = 257
    A, X, Bv = section4_problem(n, seed=61)
    LU, ipiv, Xh = lu_solve(A, Bv, K=64, algo=algo, cutoff=16)
    assert rel_residual(A, Xh, Bv) <= n * 2.0 ** -100
    _, piv_o, info = O.dd_getrf(A, pivot=True)
    assert np.array_equal(ipiv, piv_o)


# ------------------------------------- fused panel kernel (one launch per panel)
def _factor(A, K, cutoff, algo="winograd", pivot=True, form="cluster"):
    """getrf through the C ABI with the panel form restricted by
    DDG_LU_PANEL: "cluster" (thread-block cluster, the default), "grid"
    (cooperative grid) or "columns" (per-column kernels)."""
    import os
    import paper_1510_08642_gb300 as P
    old = os.environ.get("DDG_LU_PANEL")
    os.environ["DDG_LU_PANEL"] = form
    try:
        dA = to_dev(A)
        ipiv = P.getrf(dA, K=K, pivot=pivot, algo=algo, cutoff=cutoff)
        torch.cuda.synchronize()
    finally:
        if old is None:
            del os.environ["DDG_LU_PANEL"]
        else:
            os.environ["DDG_LU_PANEL"] = old
    return to_host(dA), ipiv.cpu().numpy()


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("n,K,pivot", [(1, 1, True), (37, 16, True), (300, 64, True), (1000, 256, True),
                                       (150, 32, False)])
def test_fused_panel_same_bits_as_column_steps(limbs, n, K, pivot):
    """The cluster and grid panel kernels run each column step with the
    per-column kernels' arithmetic (same quotients, same updates, same pivot
    rule), so the factors and pivots are the same bits."""
    A = I.uniform(n, n, limbs, seed=70 + n)
    if not pivot:
        A[0] += np.eye(n) * n
    LUc, pc = _factor(A, K, 16, pivot=pivot, form="columns")
    for form in ("cluster", "grid"):
        LUf, pf = _factor(A, K, 16, pivot=pivot, form=form)
        assert np.array_equal(pf, pc), form
        assert np.array_equal(LUf.view(np.uint64), LUc.view(np.uint64)), form


def _sampled_rel_residual(A, Xh, Bv, rows):
    r = O.gemm_error(np.ascontiguousarray(A[:, rows, :]), Xh, np.ascontiguousarray(Bv[:, rows, :]))
    return np.abs(r).max() / (np.abs(A[0]).sum(axis=1).max() * np.abs(Xh[0]).max())


@pytest.mark.parametrize("limbs,n,cutoff", [(2, 4096, 512), (4, 2048, 256)])
def test_bench_configs_sampled_residual_and_paths(limbs, n, cutoff):
    """The bench's LU solves (DD n = 4096, QD n = 2048, K = 256, partial
    pivoting, Winograd trailing updates): the exact residual of sampled rows
    against the oracle within n 2^-100 (DD) / n 2^-200 (QD), and the fused
    panels give the per-column kernels' factors and pivots bit for bit."""
    import paper_1510_08642_gb300 as P
    A = I.uniform(n, n, limbs, seed=71)
    X = np.zeros((limbs, n, 1))
    X[0] = 1.0
    rows = np.array(sorted({0, n - 1, *np.random.default_rng(3).choice(n, 30, replace=False)}))
    LUc, pc = _factor(A, 256, cutoff, form="columns")
    for form in ("grid", "cluster"):
        LUf, pf = _factor(A, 256, cutoff, form=form)
        assert np.array_equal(pf, pc), form
        assert np.array_equal(LUf.view(np.uint64), LUc.view(np.uint64)), form
    assert np.all(pf >= np.arange(n)) and np.all(pf < n)
    # solve b = A 1 with the factors (b from the GPU Block product, exact
    # residual of the computed x against that b)
    dA = to_dev(A)
    ones = torch.zeros((limbs, n, 1), dtype=torch.float64, device="cuda")
    ones[0] = 1.0
    b = P.gemm(dA, ones, algo="block")
    Bv = to_host(b)
    dLU = to_dev(LUf)
    P.getrs(dLU, torch.from_numpy(pf).cuda(), b)
    torch.cuda.synchronize()
    Xh = to_host(b)
    bound = n * (2.0 ** -100 if limbs == 2 else 2.0 ** -200)
    assert _sampled_rel_residual(A, Xh, Bv, rows) <= bound
