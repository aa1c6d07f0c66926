"""GPU parity for the INT8-slice DD product (algo "ozaki") through the C ABI.

* bit-exact against the oracle's restatement (oracle/ozaki.py) on small
  ragged shapes, several slice counts and all three modes: splitting,
  INT8 products and the exact recombination leave no freedom;
* within the stated bound against the exact checker, and normwise
  <= n 2^-100 on the uniform and wide-range inputs of the precision study;
* integer matrices exact.
"""
import numpy as np
import pytest

import oracle as O
import oracle.ozaki as OZ
from paper_1510_08642_gb300 import inputs as I
from tests.gpu_util import sample_entries, to_dev, to_host

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(A, B, s, C0=None, mode="set"):
    import paper_1510_08642_gb300 as P
    dC = None if C0 is None else to_dev(C0)
    C = P.gemm(to_dev(A), to_dev(B), dC, algo="ozaki", slices=s, mode=mode)
    torch.cuda.synchronize()
    return to_host(C)


@pytest.mark.parametrize("s", [2, 7, 13, 16, 18])
@pytest.mark.parametrize("shape", [(1, 1, 1), (9, 70, 13), (130, 65, 129)])
def test_bit_exact_vs_oracle(s, shape):
    m, l, n = shape
    A = I.uniform(m, l, 2, seed=30 + s)
    B = I.uniform(l, n, 2, seed=40 + s)
    got = run(A, B, s)
    want, _ = OZ.gemm(A, B, s)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("mode", ["add", "sub"])
def test_modes_bit_exact(mode):
    A = I.uniform(20, 33, 2, seed=50)
    B = I.uniform(33, 17, 2, seed=51)
    C0 = I.uniform(20, 17, 2, seed=52)
    got = run(A, B, 16, C0, mode)
    want, _ = OZ.gemm(A, B, 16, C0=C0, mode=mode)
    assert np.array_equal(got, want)


def test_wide_and_special_bit_exact():
    A = I.wide(24, 40, 2, seed=53)
    B = I.wide(40, 19, 2, seed=54)
    A[:, 3, :] = 0.0
    B[:, :, 7] *= 2.0 ** -300
    got = run(A, B, 12)
    want, _ = OZ.gemm(A, B, 12)
    assert np.array_equal(got, want)


def test_integer_exact():
    A = I.integer(70, 90, 2, seed=55, bits=20)
    B = I.integer(90, 60, 2, seed=56, bits=20)
    assert not O.gemm_error(A, B, run(A, B, 8)).any()


@pytest.mark.parametrize("kind", ["uniform", "wide"])
def test_n4096_normwise(kind):
    """The precision study's size: sampled entries, exact checker."""
    n = 4096
    gen = I.uniform if kind == "uniform" else I.wide
    A = gen(n, n, 2, seed=57)
    B = gen(n, n, 2, seed=58)
    rows, cols = sample_entries(n, n, 48, seed=59)
    for s in (13, 16):
        C = run(A, B, s)
        err = O.gemm_error(A, B, C, rows=rows, cols=cols)
        # normwise estimate from the sample: ||E||_F ~ sqrt(n^2 mean(err^2))
        est = np.sqrt(n * n * np.mean(err ** 2)) / (np.linalg.norm(A[0]) * np.linalg.norm(B[0]))
        assert est <= n * 2.0 ** -100, (s, est)
        fa = OZ.row_fields(A[0][rows], axis=1)
        fb = OZ.row_fields(B[0][:, cols], axis=0)
        scale = np.ldexp(1.0, (fa - 1022) + (fb - 1022))
        assert np.all(np.abs(err) <= (n * (s + 3) * 2.0 ** (-7 * s) + 2.0 ** -104) * scale)


def run_qd(A, B, s, C0=None, mode="set"):
    return run(A, B, s, C0, mode)


@pytest.mark.parametrize("s", [2, 9, 24, 32])
@pytest.mark.parametrize("shape", [(1, 1, 1), (9, 40, 13), (130, 65, 129)])
def test_qd_bit_exact_vs_oracle(s, shape):
    m, l, n = shape
    A = I.uniform(m, l, 4, seed=60 + s)
    B = I.uniform(l, n, 4, seed=70 + s)
    got = run_qd(A, B, s)
    want, _ = OZ.gemm(A, B, s)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("mode", ["add", "sub"])
def test_qd_modes_bit_exact(mode):
    A = I.uniform(17, 30, 4, seed=61)
    B = I.uniform(30, 11, 4, seed=62)
    C0 = I.uniform(17, 11, 4, seed=63)
    got = run_qd(A, B, 32, C0, mode)
    want, _ = OZ.gemm(A, B, 32, C0=C0, mode=mode)
    assert np.array_equal(got, want)


def test_qd_n2048_normwise_qd_accuracy():
    n = 2048
    A = I.uniform(n, n, 4, seed=64)
    B = I.uniform(n, n, 4, seed=65)
    rows, cols = sample_entries(n, n, 32, seed=66)
    C = run_qd(A, B, 32)
    err = O.gemm_error(A, B, C, rows=rows, cols=cols)
    est = np.sqrt(n * n * np.mean(err ** 2)) / (np.linalg.norm(A[0]) * np.linalg.norm(B[0]))
    assert est <= 8 * n * 2.0 ** -208, est


# ------------------------------------------------ CRT scheme (algo ozaki2) --
def run_crt(A, B, N, C0=None, mode="set"):
    import paper_1510_08642_gb300 as P
    dC = None if C0 is None else to_dev(C0)
    C = P.gemm(to_dev(A), to_dev(B), dC, algo="ozaki2", slices=N, mode=mode)
    torch.cuda.synchronize()
    return to_host(C)


@pytest.mark.parametrize("N", [2, 9, 20, 32, 40])
@pytest.mark.parametrize("shape", [(1, 1, 1), (9, 70, 13), (130, 65, 129), (200, 300, 3)])
def test_crt_bit_exact_vs_oracle(N, shape):
    """Residues, INT8 products, their reduction and the CRT reconstruction
    leave no freedom: every bit equals the oracle's exact-integer result."""
    m, l, n = shape
    A = I.uniform(m, l, 2, seed=80 + N)
    B = I.uniform(l, n, 2, seed=90 + N)
    got = run_crt(A, B, N)
    want, _ = OZ.gemm_crt(A, B, N)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("mode", ["add", "sub"])
def test_crt_modes_and_special_bit_exact(mode):
    A = I.wide(24, 40, 2, seed=81)
    B = I.wide(40, 19, 2, seed=82)
    A[:, 3, :] = 0.0
    B[:, :, 7] *= 2.0 ** -300
    C0 = I.uniform(24, 19, 2, seed=83)
    got = run_crt(A, B, 32, C0, mode)
    want, _ = OZ.gemm_crt(A, B, 32, C0=C0, mode=mode)
    assert np.array_equal(got, want)


def test_crt_integer_exact():
    A = I.integer(70, 90, 2, seed=84, bits=20)
    B = I.integer(90, 60, 2, seed=85, bits=20)
    assert not O.gemm_error(A, B, run_crt(A, B, 32)).any()


def test_crt_n4096_sampled_bit_exact_and_bound():
    """The bench's size and launch: sampled entries bit-exact against the
    oracle computed one by one, and within l 2^-P of the exact product."""
    from paper_1510_08642_gb300 import capi
    n, N = 4096, 32
    A = I.uniform(n, n, 2, seed=86)
    B = I.uniform(n, n, 2, seed=87)
    rows, cols = sample_entries(n, n, 12, seed=88)
    C = run_crt(A, B, N)
    got = C[:, rows, cols]
    want = OZ.gemm_crt_entries(A, B, N, rows, cols)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    P = capi.ddg_ozaki2_precision(N, n)
    assert P == OZ.crt_precision(N, n) == 113
    err = O.gemm_error(A, B, C, rows=rows, cols=cols)
    fa = OZ.row_fields(A[0][rows], axis=1)
    fb = OZ.row_fields(B[0][:, cols], axis=0)
    scale = np.ldexp(1.0, (fa - 1022) + (fb - 1022))
    # integer rounding of both operands, plus the final rounding of c to DD
    # (106 bits, relative to |c|, which grows like sqrt(l) here)
    assert np.all(np.abs(err) <= n * 2.0 ** -P * scale + 2.0 ** -104 * np.abs(got[0]))


def test_crt_rejects_qd_and_bad_sizes():
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    A4 = to_dev(I.uniform(8, 8, 4, seed=89))
    with pytest.raises(capi.DDGError) as e:
        P.gemm(A4, A4, algo="ozaki2")
    assert e.value.status == capi.DDG_ENOTSUP
    A2 = to_dev(I.uniform(8, 8, 2, seed=89))
    for N in (1, 41):
        with pytest.raises(capi.DDGError) as e:
            P.gemm(A2, A2, algo="ozaki2", slices=N)
        assert e.value.status == capi.DDG_EINVAL
