"""GPU parity: dd_gemm / qd_gemm through the C ABI against the CPU oracle.

* Simple (Eq. 1, k ascending, pinned DD/QD operation sequence): bit-exact
  against the oracle's triple loop on every limb of every entry.
* Block / Strassen / Winograd: error against the oracle's exact (Kulisch)
  checker within the bounds 8 l 2^-104 (Block) and 8 l^log2(12) 2^-104
  (Strassen, Winograd) normwise, 2^-208 in place of 2^-104 for QD; Block is
  also held to its elementwise bound (l + 4) u^2 sum_k |a_ik b_kj|.
* Integer matrices: every algorithm exact.
"""
import numpy as np
import pytest

import oracle as O
from paper_1510_08642_gb300 import inputs as I
from tests.gpu_util import U2, Q2, absprod, normwise_bound, sample_entries, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1510_08642_gb300 as P
    P.capi.load()


def run(A, B, C0=None, **kw):
    import paper_1510_08642_gb300 as P
    dA, dB = to_dev(A), to_dev(B)
    dC = None if C0 is None else to_dev(C0)
    dC = P.gemm(dA, dB, dC, **kw)
    torch.cuda.synchronize()
    return to_host(dC)


# ------------------------------------------------------------ Simple ------
@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("shape", [(128, 128, 128), (1, 1, 1), (7, 13, 5), (33, 65, 17), (9, 0, 4)])
def test_simple_bit_exact(limbs, shape):
    m, l, n = shape
    A = I.uniform(m, l, limbs, seed=0)
    B = I.uniform(l, n, limbs, seed=1)
    got = run(A, B, algo="simple")
    want = O.gemm_simple(A, B)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("mode", ["add", "sub"])
def test_simple_modes_bit_exact(limbs, mode):
    A = I.uniform(40, 24, limbs, seed=2)
    B = I.uniform(24, 36, limbs, seed=3)
    C0 = I.uniform(40, 36, limbs, seed=4)
    got = run(A, B, C0, algo="simple", mode=mode)
    want = O.gemm_simple(A, B, C0, mode=mode)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_simple_wide_range_bit_exact():
    A = I.wide(50, 70, 2, seed=5)
    B = I.wide(70, 30, 2, seed=6)
    assert np.array_equal(run(A, B, algo="simple"), O.gemm_simple(A, B))


# ------------------------------------------------- Block and recursion ----
CASES = [
    ("block", 64, (100, 77, 130)),
    ("block", 64, (1, 300, 1)),
    ("strassen", 64, (256, 256, 256)),
    ("winograd", 64, (256, 256, 256)),
    ("strassen", 32, (257, 255, 263)),
    ("winograd", 32, (257, 255, 263)),
    ("winograd", 16, (130, 66, 98)),
    ("winograd", 40, (200, 120, 90)),
]


def check_bounds(A, B, C, algo, C0=None, mode="set", elementwise=True):
    limbs, m, l = A.shape
    err = O.gemm_error(A, B, C, C0=C0, mode=mode)
    nw = O.normwise(err, A, B)
    assert nw <= normwise_bound(l, limbs, algo), (algo, nw)
    if algo == "block" and elementwise:
        u2 = U2 if limbs == 2 else 8 * Q2
        scale = absprod(A, B)
        bound = (2 * l + 4) * u2 * scale + (np.abs(C0[0]) * u2 * 4 if C0 is not None else 0) + 1e-300
        assert np.all(np.abs(err) <= bound)
    return nw


@pytest.mark.parametrize("accum", ["fx", "twosum"])
@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("algo,cutoff,shape", CASES)
def test_algorithms_within_bound(limbs, algo, cutoff, shape, accum):
    m, l, n = shape
    A = I.uniform(m, l, limbs, seed=7)
    B = I.uniform(l, n, limbs, seed=8)
    C = run(A, B, algo=algo, cutoff=cutoff, accum=accum)
    nw = check_bounds(A, B, C, algo)
    # far inside the bound in practice: a wrong quadrant formula is O(1)
    assert nw < (1e-28 if limbs == 2 else 1e-60)


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("algo", ["block", "strassen", "winograd"])
@pytest.mark.parametrize("mode", ["add", "sub"])
def test_update_modes(limbs, algo, mode):
    A = I.uniform(130, 98, limbs, seed=9)
    B = I.uniform(98, 66, limbs, seed=10)
    C0 = I.uniform(130, 66, limbs, seed=11)
    C = run(A, B, C0, algo=algo, cutoff=16, mode=mode)
    check_bounds(A, B, C, algo, C0=C0, mode=mode)


@pytest.mark.parametrize("accum", ["fx", "twosum"])
@pytest.mark.parametrize("algo", ["block", "strassen", "winograd"])
@pytest.mark.parametrize("limbs", [2, 4])
def test_integer_exact(algo, limbs, accum):
    m, l, n = 96, 130, 70
    A = I.integer(m, l, limbs, seed=12, bits=20)
    B = I.integer(l, n, limbs, seed=13, bits=20)
    C = run(A, B, algo=algo, cutoff=16, accum=accum)
    err = O.gemm_error(A, B, C)
    assert not err.any()


@pytest.mark.parametrize("limbs", [2, 4])
def test_pad_and_peel_agree_within_bound(limbs):
    m, l, n = 203, 181, 157
    A = I.uniform(m, l, limbs, seed=14)
    B = I.uniform(l, n, limbs, seed=15)
    for pad in (False, True):
        C = run(A, B, algo="winograd", cutoff=24, pad=pad)
        check_bounds(A, B, C, "winograd")


@pytest.mark.parametrize("algo", ["strassen", "winograd"])
def test_streams_do_not_change_bits(algo):
    A = I.uniform(300, 300, 2, seed=16)
    B = I.uniform(300, 300, 2, seed=17)
    c7 = run(A, B, algo=algo, cutoff=40, streams=7)
    c1 = run(A, B, algo=algo, cutoff=40, streams=1)
    assert np.array_equal(c7, c1)


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("accum", ["fx", "twosum"])
def test_wide_range_inputs(limbs, accum):
    A = I.wide(160, 200, limbs, seed=18)
    B = I.wide(200, 120, limbs, seed=19)
    for algo in ("block", "winograd"):
        C = run(A, B, algo=algo, cutoff=32, accum=accum)
        check_bounds(A, B, C, algo, elementwise=(algo == "block"))


@pytest.mark.parametrize("limbs", [2, 4])
def test_fx_special_values(limbs):
    """Zero rows / columns, tiny and huge magnitudes, exact cancellation."""
    m, l, n = 40, 70, 36
    A = I.uniform(m, l, limbs, seed=20)
    B = I.uniform(l, n, limbs, seed=21)
    A[:, 3, :] = 0.0            # zero row of A
    B[:, :, 5] = 0.0            # zero column of B
    A[:, 7, :] *= 2.0 ** -600   # tiny row
    B[:, :, 9] *= 2.0 ** 500    # huge column
    A[:, 11, 35:] = A[:, 11, :35]
    B[:, 35:, 13] = -B[:, :35, 13]  # row 11 x column 13 cancels exactly
    C = run(A, B, algo="block")
    err = O.gemm_error(A, B, C)
    u2 = U2 if limbs == 2 else 8 * Q2
    assert np.all(np.abs(err) <= (2 * l + 4) * u2 * absprod(A, B) + 1e-300)
    assert not C[:, 3, :].any() and not C[:, :, 5].any()


def test_paper_matrices_table1_shapes():
    """Section 3 test matrices at the Table 1 sizes, Winograd(32) and Block."""
    import tests.exact as X
    from fractions import Fraction
    s15 = X.sqrt_fraction(15)
    for n in (1023, 1024, 1025):
        A, B = I.paper_matrices(n, 2)
        for algo in ("block", "winograd", "strassen"):
            C = run(A, B, algo=algo, cutoff=32)
            rows, cols = sample_entries(n, n, 12, seed=n)
            for i, j in zip(rows, cols):
                want = s15 * (i * n * (n - 1) // 2 + (n - 1) * n * (n + 1) // 6)
                got = Fraction(float(C[0, i, j])) + Fraction(float(C[1, i, j]))
                # input rounding 2^-105 relative plus the algorithm's error
                assert abs(got - want) <= abs(want) * Fraction(1, 1 << 80)
            err = O.gemm_error(A, B, C, rows=rows, cols=cols)
            assert np.all(np.abs(err) <= normwise_bound(n, 2, algo) * absprod(A, B, rows, cols))


# ------------------------------------- narrow products (n <= 8 columns) ----
NARROW = [(300, 1000, 1), (37, 5000, 3), (130, 33, 8), (1, 1, 1), (64, 7, 5), (17, 100, 2)]


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("shape", NARROW)
def test_narrow_same_bits_as_block_tile(limbs, shape):
    """n <= 8 runs one warp per output; its window is the exact sum of the
    same truncated products the Block tile accumulates, so the result equals
    the first n columns of a product wide enough for the tile kernel."""
    m, l, n = shape
    A = I.uniform(m, l, limbs, seed=40)
    B = I.wide(l, n, limbs, seed=41)
    Bw = np.concatenate([B, I.uniform(l, 40 - n, limbs, seed=42)], axis=2)
    C = run(A, B, algo="block")
    Cw = run(A, Bw, algo="block")
    assert np.array_equal(C, Cw[:, :, :n])
    check_bounds(A, B, C, "block")


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("mode", ["add", "sub"])
def test_narrow_update_modes(limbs, mode):
    A = I.wide(200, 700, limbs, seed=43)
    B = I.uniform(700, 4, limbs, seed=44)
    C0 = I.uniform(200, 4, limbs, seed=45)
    C = run(A, B, C0, algo="winograd", cutoff=16, mode=mode)  # n <= cutoff: the base case
    check_bounds(A, B, C, "block", C0=C0, mode=mode)


@pytest.mark.parametrize("limbs", [2, 4])
def test_narrow_special_values(limbs):
    """Zero row / column, tiny and huge magnitudes, exact cancellation."""
    m, l, n = 40, 70, 6
    A = I.uniform(m, l, limbs, seed=46)
    B = I.uniform(l, n, limbs, seed=47)
    A[:, 3, :] = 0.0
    B[:, :, 5] = 0.0
    A[:, 7, :] *= 2.0 ** -600
    B[:, :, 2] *= 2.0 ** 500
    A[:, 11, 35:] = A[:, 11, :35]
    B[:, 35:, 1] = -B[:, :35, 1]  # row 11 x column 1 cancels exactly
    C = run(A, B, algo="block")
    err = O.gemm_error(A, B, C)
    u2 = U2 if limbs == 2 else 8 * Q2
    assert np.all(np.abs(err) <= (2 * l + 4) * u2 * absprod(A, B) + 1e-300)
    assert not C[:, 3, :].any() and not C[:, :, 5].any()
    assert not C[:, 11, 1].any()


def test_narrow_integer_exact():
    A = I.integer(90, 3000, 2, seed=48, bits=20)
    B = I.integer(3000, 3, 2, seed=49, bits=20)
    C = run(A, B, algo="block")
    assert not O.gemm_error(A, B, C).any()
