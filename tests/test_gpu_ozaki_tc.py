"""GPU parity for the CRT DD product on the tcgen05 tensor cores (algo
"ozaki2_tc", DDG_OZAKI2_TC) through the C ABI.

The residue products are exact integers on either engine (INT8 mma.sync
or BF16 tcgen05 with FP32 accumulation drained every 256 terms), so:

* every bit equals the oracle's exact-integer CRT result (oracle/ozaki.py)
  and the INT8 engine's result, on ragged shapes spanning several 128 x 128
  tiles, several 256-term chunks and a partial last chunk, all modes;
* residues at the extreme of their range (every residue mod 256 equal to
  -128, so every 256-term chunk sums to exactly 2^22): still exact;
* at the bench's n = 4096 and at n = 8192 with wide-range entries: sampled
  entries bit-exact against the oracle computed one by one, the error
  within l 2^-P of the row / column scale against the exact checker;
* the LU with tensor-core trailing updates: exact residual <= n 2^-100;
* no bounded device wait ran out.
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
    from paper_1510_08642_gb300 import capi
    capi.ddg_device_timeouts(reset=True)
    yield
    assert capi.ddg_device_timeouts() == 0


def run(A, B, N, algo="ozaki2_tc", C0=None, mode="set"):
    import paper_1510_08642_gb300 as P
    dC = None if C0 is None else to_dev(C0)
    C = P.gemm(to_dev(A), to_dev(B), dC, algo=algo, slices=N, mode=mode)
    torch.cuda.synchronize()
    return to_host(C)


def same_bits(a, b):
    return np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("N", [2, 9, 32, 40])
@pytest.mark.parametrize("shape", [(1, 1, 1), (9, 70, 13), (130, 65, 129), (200, 300, 3), (257, 600, 140)])
def test_tc_bit_exact_vs_oracle_and_int8(N, shape):
    m, l, n = shape
    A = I.uniform(m, l, 2, seed=180 + N)
    B = I.uniform(l, n, 2, seed=190 + N)
    got = run(A, B, N)
    want, _ = OZ.gemm_crt(A, B, N)
    assert same_bits(got, want)
    assert same_bits(got, run(A, B, N, algo="ozaki2"))


@pytest.mark.parametrize("mode", ["add", "sub"])
def test_tc_modes_and_special_bit_exact(mode):
    A = I.wide(150, 300, 2, seed=181)
    B = I.wide(300, 140, 2, seed=182)
    A[:, 3, :] = 0.0
    B[:, :, 7] *= 2.0 ** -300
    C0 = I.uniform(150, 140, 2, seed=183)
    got = run(A, B, 32, C0=C0, mode=mode)
    want, _ = OZ.gemm_crt(A, B, 32, C0=C0, mode=mode)
    assert same_bits(got, want)


def test_tc_extreme_residues_exact():
    """Entries 1/2 + (128 + 256 u) 2^-P: the scaled integers are 2^(P-1) +
    128 + 256 u, so every residue mod 256 is -128 and every product +2^14;
    each 256-term chunk of the tensor-core accumulation sums to exactly
    2^22, the edge of the exact range."""
    m, l, n, N = 130, 1024, 130, 32
    P = OZ.crt_precision(N, l)
    rng = np.random.default_rng(5)

    def operand(rows, cols):
        X = np.zeros((2, rows, cols))
        X[0] = 0.5
        u = rng.integers(0, 1 << 20, size=(rows, cols))
        X[1] = np.ldexp((128.0 + 256.0 * u), -P)
        return X
    A, B = operand(m, l), operand(l, n)
    got = run(A, B, N)
    want, _ = OZ.gemm_crt(A, B, N)
    assert same_bits(got, want)
    # operands exact at P bits: only the final rounding to DD remains
    assert np.all(np.abs(O.gemm_error(A, B, got)) <= 2.0 ** -104 * np.abs(got[0]))


def test_tc_integer_exact():
    A = I.integer(170, 390, 2, seed=184, bits=20)
    B = I.integer(390, 160, 2, seed=185, bits=20)
    assert not O.gemm_error(A, B, run(A, B, 32)).any()


@pytest.mark.parametrize("n,dist", [(4096, "uniform"), (8192, "wide")])
def test_tc_full_size_sampled_bit_exact_and_bound(n, dist):
    """The bench's sizes and launch: sampled entries bit-exact against the
    oracle computed one by one; within l 2^-P of the row / column scale."""
    N = 32
    gen = I.uniform if dist == "uniform" else I.wide
    A = gen(n, n, 2, seed=186)
    B = gen(n, n, 2, seed=187)
    rows, cols = sample_entries(n, n, 12, seed=188)
    C = run(A, B, N)
    got = C[:, rows, cols]
    want = OZ.gemm_crt_entries(A, B, N, rows, cols)
    assert same_bits(got, want)
    P = OZ.crt_precision(N, n)
    err = O.gemm_error(A, B, C, rows=rows, cols=cols)
    fa = OZ.row_fields(A[0][rows], axis=1)
    fb = OZ.row_fields(B[0][:, cols], axis=0)
    scale = np.ldexp(1.0, (fa - 1022) + (fb - 1022))
    assert np.all(np.abs(err) <= n * 2.0 ** -P * scale + 2.0 ** -104 * np.abs(got[0]))


def test_tc_lu_trailing_updates():
    import paper_1510_08642_gb300 as P
    n = 600
    A = I.uniform(n, n, 2, seed=189)
    X = np.zeros((2, n, 1))
    X[0, :, 0] = np.arange(n)
    Bv = O.gemm_simple(A, X)
    dA = to_dev(A)
    ipiv = P.getrf(dA, K=128, pivot=True, algo="ozaki2_tc", cutoff=64)
    dB = to_dev(Bv)
    P.getrs(dA, ipiv, dB)
    torch.cuda.synchronize()
    Xh = to_host(dB)
    r = O.dd_residual(A, Xh, Bv)
    rel = np.abs(r).max() / (np.abs(A[0]).sum(axis=1).max() * np.abs(Xh[0]).max())
    assert rel <= n * 2.0 ** -100


def test_tc_rejects_qd():
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    A4 = to_dev(I.uniform(8, 8, 4, seed=189))
    with pytest.raises(capi.DDGError) as e:
        P.gemm(A4, A4, algo="ozaki2_tc")
    assert e.value.status == capi.DDG_ENOTSUP
