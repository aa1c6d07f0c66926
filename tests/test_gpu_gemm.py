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


# ------------------------ operands converted once vs per staged tile ------
CONVERTED = [(100, 77, 130), (64, 32, 64), (257, 255, 263), (300, 1000, 70), (65, 33, 97)]


def _specials(A, B):
    """Zero and negative-zero rows of A, a zero column of B, subnormal leading
    limbs (lower limbs zero) in a row of A."""
    A[:, 3, :] = 0.0
    A[:, 5, :] = -0.0
    B[:, :, 7] = 0.0
    A[0, 9, :] = np.ldexp(np.arange(1, A.shape[2] + 1, dtype=np.float64), -1070)
    A[1:, 9, :] = 0.0


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("shape", CONVERTED)
def test_converted_operands_same_bits(limbs, shape):
    """Block products large enough to convert each operand once into workspace
    (accum "fx") give exactly the bits of converting every tile as it is staged
    (accum "fx_tile"), in all three modes, on wide-range operands with zeros,
    negative zeros and subnormals; and stay within the Block bounds."""
    m, l, n = shape
    A = I.wide(m, l, limbs, seed=60)
    B = I.uniform(l, n, limbs, seed=61)
    _specials(A, B)
    C0 = I.uniform(m, n, limbs, seed=62)
    for mode in ("set", "add", "sub"):
        c0 = None if mode == "set" else C0
        got = run(A, B, c0, algo="block", mode=mode)
        want = run(A, B, c0, algo="block", mode=mode, accum="fx_tile")
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), mode
        if mode == "set":
            check_bounds(A, B, got, "block")
            assert not got[:, 3, :].any() and not got[:, 5, :].any() and not got[:, :, 7].any()


@pytest.mark.parametrize("limbs", [2, 4])
@pytest.mark.parametrize("algo", ["winograd", "strassen"])
@pytest.mark.parametrize("shape", [(301, 261, 291), (200, 150, 181)])
def test_converted_leaves_same_bits(limbs, algo, shape):
    """Recursion leaves on operands converted once per node (the 14 leaf
    operands of a node in one launch): two levels with 75 x 65 x 72 leaves and
    peeled edges, and one level whose leaves (100 x 75 x 90) run on the seven
    forked streams; the same bits as the per-tile path, on both stream
    schedules."""
    m, l, n = shape
    A = I.uniform(m, l, limbs, seed=63)
    B = I.wide(l, n, limbs, seed=64)
    want = run(A, B, algo=algo, cutoff=100, accum="fx_tile")
    for streams in (7, 1):
        got = run(A, B, algo=algo, cutoff=100, streams=streams)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), streams
    check_bounds(A, B, want, algo)


def test_conversion_launches_profiled():
    """A converted Block product is two launches: the conversion of both
    operands (profile kind "convert") and the product."""
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    dA = to_dev(I.uniform(128, 96, 2, seed=65))
    dB = to_dev(I.uniform(96, 160, 2, seed=66))
    for accum, conv in (("fx", 1), ("fx_tile", 0)):
        P.gemm(dA, dB, algo="block")  # load and warm up outside the profile
        torch.cuda.synchronize()
        capi.ddg_profile_begin()
        P.gemm(dA, dB, algo="block", accum=accum)
        prof = capi.ddg_profile_end()
        assert prof["convert"]["launches"] == conv
        assert prof["convert"]["ops"] == (128 * 96 + 96 * 160 if conv else 0)
        assert prof["block"]["launches"] == 1
        assert prof["block"]["ops"] == 128 * 96 * 160


@pytest.mark.parametrize("name", ["dd_winograd_n4096", "qd_winograd_n4096", "dd_winograd_n3000",
                                  "qd_winograd_n3000"])
def test_benchmark_workload_sampled(name):
    """The benchmark's DD / QD Winograd workloads at full size (n = 4096,
    cutoff 256, seven streams, operands converted once per leaf node): sampled
    entries against the oracle's exact error within the normwise bound scaled
    elementwise, and every bit equal to the per-tile conversion path."""
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import workloads as WL
    # n = 3000: odd sizes below the top level (1500 -> 750 -> 375) peeled
    w = {x.name: x for x in (WL.DD_WINOGRAD_4096, WL.QD_WINOGRAD_4096, WL.DD_WINOGRAD_3000,
                             WL.QD_WINOGRAD_3000)}[name]
    A = I.uniform(w.n, w.n, w.limbs, seed=w.seed_a)
    B = I.uniform(w.n, w.n, w.limbs, seed=w.seed_b)
    dA, dB = to_dev(A), to_dev(B)
    C = P.gemm(dA, dB, algo=w.algo, cutoff=w.cutoff)
    Ct = P.gemm(dA, dB, algo=w.algo, cutoff=w.cutoff, accum="fx_tile")
    torch.cuda.synchronize()
    assert torch.equal(C.view(torch.int64), Ct.view(torch.int64))
    del Ct
    rows, cols = sample_entries(w.n, w.n, 60, seed=w.n + w.limbs)
    Cs = C[:, rows, cols].cpu().numpy()  # (limbs, samples)
    Cfull = np.zeros((w.limbs, w.n, w.n))
    Cfull[:, rows, cols] = Cs
    err = O.gemm_error(A, B, Cfull, rows=rows, cols=cols)
    assert np.all(np.abs(err) <= normwise_bound(w.n, w.limbs, w.algo) * absprod(A, B, rows, cols))
    # far inside the bound: a wrong quadrant formula is O(1)
    scale = absprod(A, B, rows, cols)
    assert np.all(np.abs(err) <= (1e-26 if w.limbs == 2 else 1e-58) * scale)


@pytest.mark.parametrize("algo", ["strassen", "winograd"])
def test_deep_recursion_streams_same_bits(algo):
    """Five levels with odd sizes on the way (cutoff 8: 7^5 leaves and their
    peeled edges, ~25,000 launches spread over the seven branches and issued
    round-robin): the same bits as the one-stream schedule and within the
    bound."""
    A = I.uniform(150, 146, 2, seed=20)
    B = I.uniform(146, 154, 2, seed=21)
    c7 = run(A, B, algo=algo, cutoff=8, streams=7)
    c1 = run(A, B, algo=algo, cutoff=8, streams=1)
    assert np.array_equal(c7.view(np.uint64), c1.view(np.uint64))
    rows, cols = sample_entries(150, 154, 40, seed=22)
    err = O.gemm_error(A, B, c7, rows=rows, cols=cols)
    assert np.all(np.abs(err) <= normwise_bound(146, 2, algo) * absprod(A, B, rows, cols))


@pytest.mark.parametrize("algo", ["block", "strassen", "winograd", "ozaki", "ozaki2"])
def test_empty_dimensions(algo):
    """m = 0 or n = 0: nothing is touched; l = 0: C := 0 in set mode, C
    unchanged when adding or subtracting."""
    import paper_1510_08642_gb300 as P
    for m, l, n in ((0, 5, 7), (5, 7, 0), (5, 0, 7)):
        A = to_dev(np.zeros((2, m, l)))
        B = to_dev(np.zeros((2, l, n)))
        for mode in ("set", "add", "sub"):
            C0 = I.uniform(m, n, 2, seed=23)
            dC = to_dev(C0)
            P.gemm(A, B, dC, algo=algo, cutoff=16, mode=mode)
            torch.cuda.synchronize()
            got = to_host(dC)
            want = np.zeros_like(C0) if (mode == "set" and l == 0) else C0
            assert np.array_equal(got, want), (m, l, n, mode)
