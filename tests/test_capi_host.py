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
