"""The C-ABI library builds, loads and exports every declared symbol; its
argument checks run on the host (no GPU is touched by these calls)."""
import ctypes
import re

import pytest

from paper_1510_08642_gb300 import build as B, capi

HEADER = B.INCLUDE + "/ddgemm.h"


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted({n for n in names if n not in ("if", "defined")})


def test_header_symbols_exported():
    lib = ctypes.CDLL(B.build())
    names = declared_functions()
    assert "dd_gemm" in names and "qd_gemm" in names
    for n in names:
        assert hasattr(lib, n), n
    # the binding declares a signature for every exported entry point
    assert set(names) <= set(capi.SIGNATURES), set(names) - set(capi.SIGNATURES)


def test_block_ops_per_mac():
    assert capi.ddg_block_fp64_ops_per_mac(2, 1) == 12
    assert capi.ddg_block_fp64_ops_per_mac(4, 1) == 113
    assert capi.ddg_block_fp64_ops_per_mac(2, 0) == 0
    assert capi.ddg_block_fp64_ops_per_mac(4, 0) == 0
    assert capi.ddg_block_fp64_ops_per_mac(3, 0) == -1


def test_opts_default():
    o = capi.opts()
    assert (o.algo, o.cutoff, o.pad, o.streams, o.accum, o.slices) == (capi.DDG_WINOGRAD, 512, 0, 7, 0, 0)


FAKE = 1 << 40  # never dereferenced: every call below fails validation or is empty


def _device_visible():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


# The calls below pass made-up device addresses; they are only made where no
# GPU is visible, so that a check that ever moved after a launch could not
# touch device memory through them (on a GPU the same checks are exercised
# with real tensors by the GPU tests).
no_device = pytest.mark.skipif(_device_visible(), reason="made-up device addresses: CPU-only check")


def dd(ld, base=FAKE):
    return capi.dd_mat(base, base + (1 << 30), ld)


@pytest.mark.parametrize("case,status", [
    (dict(m=-1), capi.DDG_EINVAL),
    (dict(mode=3), capi.DDG_EINVAL),
    (dict(cutoff=0), capi.DDG_EINVAL),
    (dict(streams=3), capi.DDG_EINVAL),
    (dict(pad=2), capi.DDG_EINVAL),
    (dict(lda=3), capi.DDG_EINVAL),
    (dict(nullA=True), capi.DDG_EINVAL),
    (dict(alias=True), capi.DDG_EINVAL),
    (dict(m=0), capi.DDG_OK),
    (dict(n=0), capi.DDG_OK),
])
@no_device
def test_validation(case, status):
    m, l, n = case.get("m", 8), 6, case.get("n", 5)
    A = dd(case.get("lda", 6))
    if case.get("nullA"):
        A = capi.dd_mat(0, 0, 6)
    Bm = dd(5, FAKE + (1 << 33))
    C = dd(5, FAKE + 16 if case.get("alias") else FAKE + (1 << 34))
    o = capi.opts(cutoff=case.get("cutoff", 512), pad=bool(case.get("pad", 0)), streams=case.get("streams", 7))
    if case.get("pad") == 2:
        o.pad = 2
    st = capi.dd_gemm(m, l, n, A, Bm, C, case.get("mode", 0), o, 0)
    assert st == status, capi.last_error()
    if status != capi.DDG_OK:
        assert capi.last_error()


@no_device
def test_reserved_and_accum_checked():
    o = capi.opts()
    o.reserved[0] = 1
    st = capi.dd_gemm(4, 4, 4, dd(4), dd(4, FAKE + (1 << 33)), dd(4, FAKE + (1 << 34)), 0, o, 0)
    assert st == capi.DDG_EINVAL
    for bad in (3, -1):
        o = capi.opts()
        o.accum = bad
        st = capi.dd_gemm(4, 4, 4, dd(4), dd(4, FAKE + (1 << 33)), dd(4, FAKE + (1 << 34)), 0, o, 0)
        assert st == capi.DDG_EINVAL
    assert capi.ddg_block_fp64_ops_per_mac(2, 2) == 0
    assert capi.ddg_block_fp64_ops_per_mac(2, 3) == -1


@no_device
def test_qd_validation():
    q = capi.qd_mat()
    for i in range(4):
        q.x[i] = FAKE + i * (1 << 30)
    q.ld = 2
    st = capi.qd_gemm(4, 4, 4, q, q, q, 0, None, 0)  # ld too small
    assert st == capi.DDG_EINVAL


def test_workspace_device_checked():
    # negative or too large device indices fail before any CUDA call
    lib = capi.load()
    info = capi.ddg_workspace_info()
    assert lib.ddg_workspace_reserve(-1, 1) == capi.DDG_EINVAL
    assert lib.ddg_workspace_release(64) == capi.DDG_EINVAL
    assert lib.ddg_workspace_stats(-3, ctypes.byref(info)) == capi.DDG_EINVAL
    assert lib.ddg_workspace_stats(0, None) == capi.DDG_EINVAL
    assert "workspace" in capi.last_error()


@no_device
def test_batch_arguments_checked():
    """ddg_batch_create_ex rejects bad arguments before any CUDA call."""
    lib = capi.load()
    h = ctypes.c_void_p()
    E = capi.DDG_EINVAL
    assert lib.ddg_batch_create_ex(None, 0, None, 0, 0, None) == E
    assert lib.ddg_batch_create_ex(ctypes.byref(h), -1, None, 0, 0, None) == E
    assert lib.ddg_batch_create_ex(ctypes.byref(h), 2, None, 0, 0, None) == E
    assert lib.ddg_batch_create_ex(ctypes.byref(h), 0, None, 2, 0, None) == E
    assert "use_graph" in capi.last_error()
    assert lib.ddg_batch_create_ex(ctypes.byref(h), 0, None, 0, 2, None) == E
    assert "flags" in capi.last_error()
    assert not h.value

    def prob(**kw):
        p = capi.ddg_problem()
        p.limbs, p.mode, p.m, p.l, p.n = 2, 0, 8, 6, 5
        p.algo, p.cutoff = capi.DDG_WINOGRAD, 64
        for q in range(2):
            p.A[q], p.B[q], p.C[q] = FAKE + q * (1 << 30), FAKE + (1 << 33) + q * (1 << 30), FAKE + (1 << 34) + q * (1 << 30)
        p.lda, p.ldb, p.ldc = 6, 5, 5
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    for kw, why in ((dict(limbs=3), "limbs"), (dict(m=-1), "negative"), (dict(mode=5), "mode"),
                    (dict(algo=capi.DDG_SIMPLE), "algo"), (dict(cutoff=0), "cutoff"),
                    (dict(lda=5), "ld too small"), (dict(ldc=4), "ld too small")):
        probs = (capi.ddg_problem * 2)(prob(), prob(**kw))
        assert lib.ddg_batch_create_ex(ctypes.byref(h), 2, probs, 0, 0, None) == E, kw
        err = capi.last_error()
        assert err.startswith("problem 1: ") and why in err, (kw, err)
        assert not h.value


@no_device
def test_lu_arguments_checked():
    """dd_getrf / dd_getrs / qd_getrf / qd_getrs reject bad arguments (and
    return at once for n = 0) before any CUDA call."""
    lib = capi.load()
    E, OK = capi.DDG_EINVAL, capi.DDG_OK
    A = dd(8)
    piv = ctypes.c_void_p(FAKE + (1 << 35))
    o = capi.opts()

    def getrf(n=8, A=A, ipiv=piv, K=4, pivot=1, opts=o):
        return lib.dd_getrf(n, A, ipiv, K, pivot, ctypes.byref(opts) if opts is not None else None, None, None)

    for kw, why in ((dict(n=-1), "negative"), (dict(K=0), "K"), (dict(K=513), "K"),
                    (dict(pivot=2), "pivot"), (dict(A=capi.dd_mat(0, 0, 8)), "null plane"),
                    (dict(A=dd(7)), "ld"), (dict(ipiv=None), "ipiv")):
        assert getrf(**kw) == E, kw
        assert capi.last_error().startswith("dd_getrf: ") and why in capi.last_error(), (kw, capi.last_error())
    for field, bad in (("algo", 9), ("cutoff", 0), ("accum", 3), ("pad", 2), ("streams", 3)):
        ob = capi.opts()
        setattr(ob, field, bad)
        assert getrf(opts=ob) == E and "invalid options" in capi.last_error(), field
    assert getrf(n=0, ipiv=None) == OK and getrf(n=0, opts=None) == OK

    Bm = dd(1, FAKE + (1 << 36))
    assert lib.dd_getrs(8, -1, A, piv, Bm, None) == E
    assert lib.dd_getrs(8, 1, A, None, Bm, None) == E and "ipiv" in capi.last_error()
    assert lib.dd_getrs(8, 2, A, piv, Bm, None) == E and "ld" in capi.last_error()
    assert lib.dd_getrs(8, 1, A, piv, capi.dd_mat(0, 0, 1), None) == E
    assert lib.dd_getrs(0, 1, A, None, Bm, None) == OK
    assert lib.dd_getrs(8, 0, A, piv, Bm, None) == OK

    q = capi.qd_mat()
    for i in range(4):
        q.x[i] = FAKE + i * (1 << 30)
    q.ld = 8
    assert lib.qd_getrf(8, q, piv, 0, 1, None, None, None) == E and capi.last_error().startswith("qd_getrf")
    q.x[3] = 0
    assert lib.qd_getrf(8, q, piv, 4, 1, None, None, None) == E and "null plane" in capi.last_error()
    assert lib.qd_getrs(8, 1, q, piv, q, None) == E and capi.last_error().startswith("qd_getrs")


@no_device
def test_batch_problem_overlap_checked():
    """A batch problem whose C overlaps its own A or B is refused, like
    dd_gemm; views of one matrix that share no element are accepted."""
    lib = capi.load()
    h = ctypes.c_void_p()
    M = FAKE  # one made-up 16 x 16 DD matrix (planes 1 GiB apart), ld 16

    def prob(a_col, c_col, m=8, l=4, n=4):
        p = capi.ddg_problem()
        p.limbs, p.mode, p.m, p.l, p.n = 2, 0, m, l, n
        p.algo, p.cutoff = capi.DDG_BLOCK, 64
        for q in range(2):
            p.A[q] = M + q * (1 << 30) + 8 * a_col
            p.B[q] = FAKE + (1 << 33) + q * (1 << 30)
            p.C[q] = M + q * (1 << 30) + 8 * c_col
        p.lda = p.ldc = 16
        p.ldb = n
        return p

    # C in columns 2..5 overlaps A in columns 0..3 of the same rows
    probs = (capi.ddg_problem * 1)(prob(0, 2))
    assert lib.ddg_batch_create_ex(ctypes.byref(h), 1, probs, 0, 0, None) == capi.DDG_EINVAL
    assert "problem 0: C overlaps A or B" in capi.last_error()
    # C in columns 4..7 and A in columns 0..3: interleaved rows, no shared element
    probs = (capi.ddg_problem * 1)(prob(0, 4))
    lib.ddg_batch_create_ex(ctypes.byref(h), 1, probs, 0, 0, None)
    assert not capi.last_error().startswith("problem"), capi.last_error()
    # C's lo plane on A's hi plane
    p = prob(0, 4)
    p.C[1] = p.A[0]
    probs = (capi.ddg_problem * 1)(p)
    assert lib.ddg_batch_create_ex(ctypes.byref(h), 1, probs, 0, 0, None) == capi.DDG_EINVAL
    assert "C overlaps A or B" in capi.last_error()
