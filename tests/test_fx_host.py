"""Host checks of the Block kernel's fixed-point helpers (fx.cuh), compiled
for the CPU with nvcc and compared with exact integer arithmetic:

* to_fixed: the W-word integer M of a DD / QD number equals the exact sum
  of its limbs at the scale of the leading limb, truncated below bit 0
  (at most one unit per lower limb), with the leading limb's sign;
* mul_top: the kept words of a b lie within (D + 1) 2^32 units below
  floor(a b / 2^(32 D));
* place_shr: the window gains exactly sign * floor(p / 2^sh) (mod 2^(32 NW)),
  on the two fast-path offsets and the general path;
* acc_mag_below: the rescue test of the Block epilogue, |A| < 2^bits for a
  two's-complement window, at and around the threshold and for both signs.
"""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "fx_check.cu")
CSRC = os.path.join(ROOT, "paper_1510_08642_gb300", "csrc")


@pytest.fixture(scope="module")
def fxbin(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("fx") / "fx_check")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-o", out, SRC])
    return out


def run(binary, lines):
    r = subprocess.run([binary], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return r.stdout.strip().splitlines()


def hexd(x):
    return "%016x" % struct.unpack("<Q", struct.pack("<d", x))[0]


def words(v, n):
    return [(v >> (32 * i)) & 0xFFFFFFFF for i in range(n)]


def value(ws):
    return sum(w << (32 * i) for i, w in enumerate(ws))


def expansion(rng, L, sparse=False):
    x = [math.ldexp(rng.random() + 0.5, rng.randint(-40, 40)) * rng.choice([-1, 1])]
    for _ in range(L - 1):
        gap = rng.choice([53, 54, 60, 90, 200]) if sparse else 53
        x.append(x[-1] * 2.0 ** -gap * (rng.random() - 0.5) if rng.random() < 0.9 else 0.0)
    # renormalise with exact rationals: greedy nearest doubles
    v = sum(Fraction(t) for t in x)
    out = []
    for _ in range(L):
        d = float(v)
        out.append(d)
        v -= Fraction(d)
    return out


@pytest.mark.parametrize("L,W", [(2, 4), (4, 7)])
def test_to_fixed_exact_up_to_truncation(fxbin, L, W):
    rng = random.Random(L)
    cases = [expansion(rng, L, sparse=(i % 3 == 0)) for i in range(400)]
    cases += [[0.0] * L, [1.0] + [0.0] * (L - 1), [-(2.0 ** 1023)] + [0.0] * (L - 1),
              [5e-324] + [0.0] * (L - 1), [1.0, -2.0 ** -54] + [0.0] * (L - 2)]
    out = run(fxbin, [f"T {L} " + " ".join(hexd(t) for t in x) for x in cases])
    for x, line in zip(cases, out):
        vals = [int(t) for t in line.split()]
        es, M = vals[0], value(vals[1:])
        exact = sum(Fraction(t) for t in x)
        if x[0] == 0.0:
            assert M == 0
            continue
        f, s = es & 0xFFFF, es >> 16
        assert s == (1 if x[0] < 0 else 0)
        assert M < 2 ** (32 * W)
        unit = Fraction(2) ** (max(f, 1) - 1075 - (32 * W - 53))
        got = M * unit
        diff = abs(exact) - got
        assert -(L - 1) * unit <= diff <= (L - 1) * unit, (x, float(diff / unit))


@pytest.mark.parametrize("W,D", [(4, 3), (7, 6)])
def test_mul_top_within_dropped_columns(fxbin, W, D):
    rng = random.Random(W)
    cases = [(rng.getrandbits(32 * W), rng.getrandbits(32 * W)) for _ in range(300)]
    cases += [(2 ** (32 * W) - 1, 2 ** (32 * W) - 1), (0, 12345), (1 << (32 * W - 1), 3)]
    lines = [f"M {W} {D} " + " ".join(map(str, words(a, W) + words(b, W))) for a, b in cases]
    for (a, b), line in zip(cases, run(fxbin, lines)):
        p = value([int(t) for t in line.split()])
        exact = (a * b) >> (32 * D)
        assert 0 <= exact - p < (D + 1) * 2 ** 32


@pytest.mark.parametrize("W", [4, 7])
def test_mul_top_hi_is_its_definition(fxbin, W):
    """mul_top_hi: the words at columns W .. 2W-1 of the sum of the partial
    products a_i b_j with i + j >= W plus the high halves of those with
    i + j = W - 1 (exact big-integer sum, written out here); below
    floor(a b / 2^(32 W)) by less than 2 W (the dropped column W - 1)."""
    rng = random.Random(100 + W)
    cases = [(rng.getrandbits(32 * W), rng.getrandbits(32 * W)) for _ in range(300)]
    cases += [(2 ** (32 * W) - 1, 2 ** (32 * W) - 1), (0, 12345), (1 << (32 * W - 1), 3), (2 ** 64 - 1, 2 ** 96 + 7)]
    lines = [f"H {W} " + " ".join(map(str, words(a, W) + words(b, W))) for a, b in cases]
    for (a, b), line in zip(cases, run(fxbin, lines)):
        q = value([int(t) for t in line.split()])
        aw, bw = words(a, W), words(b, W)
        s = 0
        for i in range(W):
            for j in range(W):
                pr = aw[i] * bw[j]
                if i + j >= W:
                    s += pr << (32 * (i + j))
                elif i + j == W - 1:
                    s += (pr >> 32) << (32 * W)
        assert q == s >> (32 * W)
        exact = (a * b) >> (32 * W)
        assert 0 <= exact - q < 2 * W


@pytest.mark.parametrize("L", [2, 4])
def test_pre_shifted_term_within_its_bound(fxbin, L):
    """The pre-shifted form's term (fx_pre.cuh: operands shifted to the
    row / column fields fa, fb, fx::mul_top_hi, the sign) against the exact
    product, in window units 2^(fa + fb + LSB0): below 2^35.33 (DD) / 2^36
    (QD) units, the bound the acceptance test at 2^142 / 2^245 units turns
    into the elementwise bound; zero for small integers within 64 bits of
    their maxima (both errors vanish there)."""
    rng = random.Random(200 + L)
    NW, lsb0, bound = (6, -2204, 2.0 ** 35.33) if L == 2 else (9, -2300, 2.0 ** 36)
    field = lambda x: max(1, (struct.unpack("<Q", struct.pack("<d", x[0]))[0] >> 52) & 0x7FF)  # noqa: E731
    cases, lines = [], []
    for t in range(600):
        xa, xb = expansion(rng, L, sparse=t % 3 == 0), expansion(rng, L, sparse=t % 5 == 0)
        fa = field(xa) + rng.choice([0, 0, 1, 3, 17, 40, 90, 130, 300])
        fb = field(xb) + rng.choice([0, 0, 2, 5, 31, 64, 100, 230])
        cases.append((xa, xb, fa, fb))
    for t in range(100):  # small integers within 64 bits of their maxima: exact
        a, b = rng.randint(-2 ** 20, 2 ** 20) or 1, rng.randint(-2 ** 20, 2 ** 20) or 1
        xa, xb = [float(a)] + [0.0] * (L - 1), [float(b)] + [0.0] * (L - 1)
        cases.append((xa, xb, field(xa) + rng.randint(0, 40), field(xb) + rng.randint(0, 20)))
    for xa, xb, fa, fb in cases:
        lines.append(f"S {L} {fa} {fb} " + " ".join(hexd(v) for v in xa + xb))
    for k, ((xa, xb, fa, fb), line) in enumerate(zip(cases, run(fxbin, lines))):
        w = value([int(v) for v in line.split()])
        if w >= 1 << (32 * NW - 1):
            w -= 1 << (32 * NW)
        exact = sum(Fraction(v) for v in xa) * sum(Fraction(v) for v in xb) / Fraction(2) ** (fa + fb + lsb0)
        err = abs(Fraction(w) - exact)
        assert err < bound, (k, float(err))
        if k >= 600:
            assert err == 0, (k, xa[0], xb[0], fa, fb)


@pytest.mark.parametrize("NW,K", [(6, 5), (9, 8)])
def test_place_shr_exact(fxbin, NW, K):
    rng = random.Random(NW)
    cases = []
    for i in range(400):
        sh = rng.choice([0, 1, 31, 32, 33, 63, 64, 65, 95, 127, 32 * K - 1, 32 * K, 32 * K + 40,
                         rng.randint(0, 40 * K)])
        cases.append((sh, rng.randint(0, 1), rng.getrandbits(32 * NW - 2), rng.getrandbits(32 * K)))
    lines = [f"P {NW} {K} {sh} {neg} " + " ".join(map(str, words(acc, NW) + words(p, K)))
             for sh, neg, acc, p in cases]
    mod = 2 ** (32 * NW)
    for (sh, neg, acc, p), line in zip(cases, run(fxbin, lines)):
        got = value([int(t) for t in line.split()])
        want = (acc + (-(p >> sh) if neg else (p >> sh))) % mod
        assert got == want, (sh, neg)


def unhex(h):
    return struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0]


def limb_contrib(x, emax, top):
    """x 2^(top - (emax - 1075)) truncated toward zero, as an exact integer."""
    if x == 0.0:
        return 0
    fr = Fraction(x) * Fraction(2) ** (top - (emax - 1075))
    return int(fr)  # truncation toward zero


@pytest.mark.parametrize("L,NW", [(2, 5), (4, 9)])
def test_exact_sums_and_rounding_back(fxbin, L, NW):
    """add_at places every limb exactly (truncated below the common unit);
    from_fixed returns the expansion nearest the sum: for DD hi = sum rounded
    to 53 bits and |lo| <= ulp(hi) / 2; the expansion's value is within
    2^-(53 L - 1) of the sum."""
    rng = random.Random(10 + L)
    top = 32 * NW - 58
    lines, cases = [], []
    for i in range(300):
        n = rng.randint(1, 7)
        xs = [expansion(rng, L, sparse=(i % 4 == 0)) for _ in range(n)]
        if i % 5 == 0 and n >= 2:  # heavy cancellation
            xs[1] = [-t for t in xs[0]]
            xs[1][L - 1] = xs[1][L - 1] * 0.5
        sg = [rng.randint(0, 1) for _ in range(n)]
        emax = max(max(1, (struct.unpack("<Q", struct.pack("<d", x[0]))[0] >> 52) & 0x7FF) for x in xs)
        cases.append((xs, sg, emax))
        lines.append(f"A {L} {emax} {top} {n} " + " ".join(
            f"{s_} " + " ".join(hexd(t) for t in x) for x, s_ in zip(xs, sg)))
    mod = 2 ** (32 * NW)
    for (xs, sg, emax), line in zip(cases, run(fxbin, lines)):
        vw, limbs = line.split(";")
        V = value([int(t) for t in vw.split()])
        want = sum((-1 if s_ else 1) * limb_contrib(t, emax, top) for x, s_ in zip(xs, sg) for t in x)
        assert V == want % mod
        Vs = V - mod if V >= mod // 2 else V
        exact = Fraction(Vs) * Fraction(2) ** (emax - 1075 - top)
        out = [unhex(h) for h in limbs.split()]
        got = sum(Fraction(t) for t in out)
        if exact == 0:
            assert got == 0
            continue
        assert abs(got - exact) <= abs(exact) * Fraction(1, 2 ** (53 * L - 1))
        hi = Fraction(out[0])
        ulp = Fraction(2) ** (math.frexp(out[0])[1] - 53)
        assert abs(exact - hi) <= ulp / 2 + abs(exact) * Fraction(1, 2 ** 150)
        if L == 2:
            assert abs(Fraction(out[1])) <= ulp / 2


@pytest.mark.parametrize("NW,W", [(6, 4), (9, 7)])
def test_normalize_and_arithmetic_shift(fxbin, NW, W):
    """acc_normalize: leading one found and moved to bit 32 W - 1, the W
    words are the leading bits (truncated); acc_sar: floor(A / 2^s) for a
    two's-complement A."""
    rng = random.Random(NW)
    cases = [rng.getrandbits(rng.randint(1, 32 * NW - 1)) for _ in range(300)] + [0, 1, 2 ** (32 * NW - 1) - 1]
    out = run(fxbin, [f"N {NW} {W} " + " ".join(map(str, words(a, NW))) for a in cases])
    for a, line in zip(cases, out):
        vals = [int(t) for t in line.split()]
        p, M = vals[0], value(vals[1:])
        if a == 0:
            assert p == -1 and M == 0
            continue
        assert p == a.bit_length() - 1
        sh = (32 * W - 1) - p
        assert M == (a << sh if sh >= 0 else a >> -sh) % 2 ** (32 * W)
    mod = 2 ** (32 * NW)
    sc = [(rng.choice([0, 1, 5, 31, 32, 33, 64, 100, 32 * NW - 1, 32 * NW + 7]), rng.getrandbits(32 * NW)) for _ in range(300)]
    out = run(fxbin, [f"R {NW} {s} " + " ".join(map(str, words(a, NW))) for s, a in sc])
    for (s, a), line in zip(sc, out):
        got = value([int(t) for t in line.split()])
        signed = a - mod if a >= mod // 2 else a
        assert got == (signed >> s) % mod


@pytest.mark.parametrize("L,W", [(2, 4), (4, 7)])
def test_operand_to_limbs_canonical(fxbin, L, W):
    """operand_to_limbs: greedy round-to-nearest limbs of M 2^(e - 1075 -
    (32 W - 53)): each limb is the remaining value rounded to 53 bits, so
    |limb_{q+1}| <= ulp(limb_q) / 2 and the sum is within half an ulp of the
    last limb of the exact value."""
    rng = random.Random(20 + L)
    cases = []
    for i in range(300):
        M = rng.getrandbits(32 * W - 1) | (1 << (32 * W - 1))
        if i % 4 == 0:  # long runs of zeros / ones below the leading bits
            M = (1 << (32 * W - 1)) | (rng.getrandbits(20) << rng.randint(0, 32 * W - 30))
        if i % 7 == 0:
            M = (2 ** (32 * W) - 1) ^ rng.getrandbits(8)
        cases.append((M, rng.randint(900, 1100), rng.randint(0, 1)))
    out = run(fxbin, [f"O {L} {e} {s_} " + " ".join(map(str, words(M, W))) for M, e, s_ in cases])
    for (M, e, s_), line in zip(cases, out):
        limbs = [unhex(h) for h in line.split()]
        exact = Fraction(M) * Fraction(2) ** (e - 1075 - (32 * W - 53)) * (-1 if s_ else 1)
        rem = exact
        for q, x in enumerate(limbs):
            if x == 0.0:
                assert all(t == 0.0 for t in limbs[q:])
                break
            ulp = Fraction(2) ** (math.frexp(x)[1] - 53)
            assert abs(rem - Fraction(x)) <= ulp / 2, (q, M)
            rem -= Fraction(x)
        assert abs(rem) <= abs(exact) * Fraction(1, 2 ** (53 * L - 1))


def test_qd_reciprocal_refinement(fxbin):
    """qd_recip_refine (the LU's QD pivot reciprocal): from a DD
    approximation the result is within 2^-208 of 1/b and canonical."""
    rng = random.Random(33)
    cases = []
    for i in range(200):
        b = expansion(rng, 4, sparse=(i % 3 == 0))
        if i % 10 == 0:
            b = [float(rng.randint(1, 1000)) * rng.choice([-1, 1]), 0.0, 0.0, 0.0]
        exact = 1 / sum(Fraction(t) for t in b)
        y0 = float(exact)
        y1 = float(exact - Fraction(y0))
        if i % 5 == 0:  # a double-only start (~53 bits)
            y1 = 0.0
        cases.append((b, exact, y0, y1))
    out = run(fxbin, ["Q " + " ".join(hexd(t) for t in b) + f" {hexd(y0)} {hexd(y1)}" for b, _, y0, y1 in cases])
    for (b, exact, _, _), line in zip(cases, out):
        r = [unhex(h) for h in line.split()]
        got = sum(Fraction(t) for t in r)
        assert abs(got - exact) <= abs(exact) * Fraction(1, 2 ** 208), b
        for q in range(3):
            if r[q + 1] != 0.0:
                assert abs(r[q + 1]) <= 2.0 ** (math.frexp(r[q])[1] - 54)


@pytest.mark.parametrize("L", [2, 4])
def test_window_multiply_subtract(fxbin, L):
    """x - l y in a window (the LU's column update and triangular-solve
    step): one rounding of the exact value plus 2^-120 (DD) / 2^-216 (QD)
    of max(|x|, |l y|), including the window moving up for a large product
    and cancellation."""
    rng = random.Random(40 + L)
    cases = []
    for i in range(300):
        x, l, y = (expansion(rng, L, sparse=(i % 3 == 0)) for _ in range(3))
        if i % 4 == 0:
            x = [t * 2.0 ** -60 for t in x]  # product far above x: window moves up
        if i % 5 == 0:  # cancellation: x ~ l y
            p = sum(Fraction(t) for t in l) * sum(Fraction(t) for t in y)
            x = [float(p)] + [0.0] * (L - 1)
        if i % 11 == 0:
            l = [0.0] * L
        cases.append((x, l, y))
    out = run(fxbin, [f"F {L} " + " ".join(hexd(t) for t in x + l + y) for x, l, y in cases])
    for (x, l, y), line in zip(cases, out):
        r = [unhex(h) for h in line.split()]
        X = sum(Fraction(t) for t in x)
        P = sum(Fraction(t) for t in l) * sum(Fraction(t) for t in y)
        exact = X - P
        scale = max(abs(X), abs(P))
        got = sum(Fraction(t) for t in r)
        # one rounding to L limbs, plus the dropped partial products of the
        # W-word product (2^-123 / 2^-219 of |l y|) and the window's floor
        slack = Fraction(1, 2 ** (120 if L == 2 else 216))
        assert abs(got - exact) <= abs(exact) * Fraction(1, 2 ** (53 * L - 1)) + scale * slack, (x, l, y)


@pytest.mark.parametrize("NW,bits", [(6, 106), (9, 212), (6, 32), (9, 31)])
def test_acc_mag_below_threshold(fxbin, NW, bits):
    """|A| < 2^bits exactly, for values on both sides of 2^bits, both signs,
    zero and the window's extremes (two's complement, NW words)."""
    rng = random.Random(NW * 1000 + bits)
    mags = [0, 1, (1 << bits) - 1, 1 << bits, (1 << bits) + 1, (1 << (bits - 1)),
            (1 << (32 * NW - 2)), (1 << (32 * NW - 1)) - 1]
    mags += [rng.getrandbits(rng.randint(1, 32 * NW - 2)) for _ in range(300)]
    vals = [v for m in mags for v in (m, -m)]
    lines = [f"B {NW} {bits} " + " ".join(str(w) for w in words(v % (1 << (32 * NW)), NW)) for v in vals]
    out = run(fxbin, lines)
    for v, o in zip(vals, out):
        assert int(o) == (1 if abs(v) < (1 << bits) else 0), (v, bits)
