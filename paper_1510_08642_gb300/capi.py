"""ctypes binding of the C ABI in include/ddgemm.h (argument marshalling only).

Every step of a product runs in the CUDA library libddgemm.so; this module
only converts Python arguments to the C structures. There is no fallback:
if the library is missing or fails to load, calls raise.

Names follow the header: dd_gemm, qd_gemm, ddg_opts_default, ddg_last_error,
ddg_block_fp64_ops_per_mac; the structures dd_mat, qd_mat and ddg_opts.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_i32, c_i64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p

DDG_OK, DDG_EINVAL, DDG_ENOMEM, DDG_ECUDA, DDG_ESINGULAR, DDG_ETIMEOUT, DDG_ENOTSUP = range(7)
STATUS_NAMES = ["DDG_OK", "DDG_EINVAL", "DDG_ENOMEM", "DDG_ECUDA", "DDG_ESINGULAR",
                "DDG_ETIMEOUT", "DDG_ENOTSUP"]
DDG_SIMPLE, DDG_BLOCK, DDG_STRASSEN, DDG_WINOGRAD, DDG_OZAKI, DDG_OZAKI2, DDG_OZAKI2_TC = range(7)
ALGOS = {"simple": DDG_SIMPLE, "block": DDG_BLOCK, "strassen": DDG_STRASSEN,
         "winograd": DDG_WINOGRAD, "ozaki": DDG_OZAKI, "ozaki2": DDG_OZAKI2, "ozaki2_tc": DDG_OZAKI2_TC}
DDG_SET, DDG_ADD, DDG_SUB = range(3)
MODES = {"set": DDG_SET, "add": DDG_ADD, "sub": DDG_SUB}


class dd_mat(ctypes.Structure):
    _fields_ = [("hi", c_vp), ("lo", c_vp), ("ld", c_i64)]


class qd_mat(ctypes.Structure):
    _fields_ = [("x", c_vp * 4), ("ld", c_i64)]


class ddg_opts(ctypes.Structure):
    _fields_ = [("algo", c_i32), ("cutoff", c_i32), ("pad", c_i32), ("streams", c_i32),
                ("accum", c_i32), ("slices", c_i32), ("reserved", c_i32 * 2)]


class ddg_kernel_prof(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("sum_ms", ctypes.c_double),
                ("busy_ms", ctypes.c_double), ("ops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


PROF_KINDS = ("simple", "block", "pass", "ozaki", "gemv", "convert", "tensor")


class ddg_problem(ctypes.Structure):
    _fields_ = [("limbs", c_i32), ("mode", c_i32), ("m", c_i64), ("l", c_i64), ("n", c_i64),
                ("A", c_vp * 4), ("lda", c_i64), ("B", c_vp * 4), ("ldb", c_i64),
                ("C", c_vp * 4), ("ldc", c_i64), ("algo", c_i32), ("cutoff", c_i32)]


class ddg_batch_stats(ctypes.Structure):
    _fields_ = [("problems", c_i64), ("leaf_tasks", c_i64), ("leaf_tiles", c_i64),
                ("pass_tasks", c_i64), ("launches_per_run", c_i64),
                ("workspace_bytes", ctypes.c_uint64), ("leaf_macs", ctypes.c_double)]


class ddg_workspace_info(ctypes.Structure):
    _fields_ = [("reserved_bytes", ctypes.c_uint64), ("used_bytes", ctypes.c_uint64),
                ("threshold_bytes", ctypes.c_uint64), ("used_high_bytes", ctypes.c_uint64)]


class DDGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


# Every exported symbol and its ctypes signature (restype, argtypes).
SIGNATURES = {
    "ddg_opts_default": (None, [ctypes.POINTER(ddg_opts)]),
    "dd_gemm": (c_i32, [c_i64, c_i64, c_i64, dd_mat, dd_mat, dd_mat, c_i32,
                        ctypes.POINTER(ddg_opts), c_vp]),
    "qd_gemm": (c_i32, [c_i64, c_i64, c_i64, qd_mat, qd_mat, qd_mat, c_i32,
                        ctypes.POINTER(ddg_opts), c_vp]),
    "dd_gemm_noalloc": (c_i32, [c_i64, c_i64, c_i64, dd_mat, dd_mat, dd_mat, c_i32,
                                ctypes.POINTER(ddg_opts), c_vp]),
    "ddg_block_fp64_ops_per_mac": (c_i32, [c_i32, c_i32]),
    "ddg_ozaki2_precision": (c_i32, [c_i32, c_i64]),
    "ddg_batch_create": (c_i32, [ctypes.POINTER(c_vp), c_i32, ctypes.POINTER(ddg_problem), c_i32, c_vp]),
    "ddg_batch_create_ex": (c_i32, [ctypes.POINTER(c_vp), c_i32, ctypes.POINTER(ddg_problem), c_i32, c_i32,
                                    c_vp]),
    "ddg_batch_run": (c_i32, [c_vp, c_vp]),
    "ddg_batch_get_stats": (c_i32, [c_vp, ctypes.POINTER(ddg_batch_stats)]),
    "ddg_batch_destroy": (c_i32, [c_vp, c_vp]),
    "dd_gemm_batched": (c_i32, [c_i32, ctypes.POINTER(ddg_problem), c_vp]),
    "dd_getrf": (c_i32, [c_i64, dd_mat, c_vp, c_i32, c_i32, ctypes.POINTER(ddg_opts), c_vp, c_vp]),
    "dd_getrs": (c_i32, [c_i64, c_i64, dd_mat, c_vp, dd_mat, c_vp]),
    "qd_getrf": (c_i32, [c_i64, qd_mat, c_vp, c_i32, c_i32, ctypes.POINTER(ddg_opts), c_vp, c_vp]),
    "qd_getrs": (c_i32, [c_i64, c_i64, qd_mat, c_vp, qd_mat, c_vp]),
    "ddg_workspace_reserve": (c_i32, [c_i32, ctypes.c_uint64]),
    "ddg_workspace_release": (c_i32, [c_i32]),
    "ddg_workspace_stats": (c_i32, [c_i32, ctypes.POINTER(ddg_workspace_info)]),
    "ddg_last_error": (ctypes.c_char_p, []),
    "ddg_kernel_launches": (ctypes.c_uint64, []),
    "ddg_device_timeouts": (c_i32, [c_i32]),
    "ddg_test_bounded_wait": (c_i32, [c_i32]),
    "ddg_profile_begin": (c_i32, []),
    "ddg_profile_end": (c_i32, [ctypes.POINTER(ddg_kernel_prof), c_i32]),
}

_lib = None


def load(path: str | None = None):
    """Load libddgemm.so (building it first if absent); raises if impossible."""
    global _lib
    if _lib is None:
        p = path or _build.LIB_PATH
        if not os.path.exists(p):
            _build.build()
        L = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return load().ddg_last_error().decode()


def check(status: int) -> None:
    if status != DDG_OK:
        raise DDGError(status, last_error())


ACCUMS = {"fx": 0, "twosum": 1, "fx_tile": 2}


def opts(algo="winograd", cutoff: int = 512, pad: bool = False, streams: int = 7,
         accum="fx", slices: int = 0) -> ddg_opts:
    o = ddg_opts()
    load().ddg_opts_default(ctypes.byref(o))
    o.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    o.cutoff = int(cutoff)
    o.pad = 1 if pad else 0
    o.streams = int(streams)
    o.accum = ACCUMS[accum] if isinstance(accum, str) else int(accum)
    o.slices = int(slices)
    return o


def dd_gemm(m, l, n, A: dd_mat, B: dd_mat, C: dd_mat, mode: int, o: ddg_opts | None,
            stream: int = 0) -> int:
    return load().dd_gemm(m, l, n, A, B, C, mode, ctypes.byref(o) if o is not None else None,
                          c_vp(stream))


def qd_gemm(m, l, n, A: qd_mat, B: qd_mat, C: qd_mat, mode: int, o: ddg_opts | None,
            stream: int = 0) -> int:
    return load().qd_gemm(m, l, n, A, B, C, mode, ctypes.byref(o) if o is not None else None,
                          c_vp(stream))


def dd_gemm_noalloc(m, l, n, A: dd_mat, B: dd_mat, C: dd_mat, mode: int, o: ddg_opts | None,
                    stream: int = 0) -> int:
    """dd_gemm with its temporaries in the library's fixed 64 MiB array."""
    return load().dd_gemm_noalloc(m, l, n, A, B, C, mode,
                                  ctypes.byref(o) if o is not None else None, c_vp(stream))


def ddg_block_fp64_ops_per_mac(limbs: int, accum: int = 0) -> int:
    return load().ddg_block_fp64_ops_per_mac(limbs, accum)


def ddg_ozaki2_precision(moduli: int, l: int) -> int:
    return load().ddg_ozaki2_precision(moduli, l)


def ddg_kernel_launches() -> int:
    return load().ddg_kernel_launches()


def ddg_device_timeouts(reset: bool = False) -> int:
    return load().ddg_device_timeouts(1 if reset else 0)


def ddg_test_bounded_wait(which: int) -> int:
    return load().ddg_test_bounded_wait(which)


def ddg_profile_begin() -> None:
    check(load().ddg_profile_begin())


def ddg_profile_end() -> dict:
    """Per kernel kind: launches, sum_ms, busy_ms, ops (see ddg_kernel_prof), bytes."""
    arr = (ddg_kernel_prof * len(PROF_KINDS))()
    check(load().ddg_profile_end(arr, len(PROF_KINDS)))
    return {k: {f: getattr(arr[i], f) for f, _ in ddg_kernel_prof._fields_}
            for i, k in enumerate(PROF_KINDS)}


def dd_getrf(n, A: dd_mat, ipiv: int, K: int, pivot: int, o: ddg_opts | None, info: int | None,
             stream: int = 0) -> int:
    return load().dd_getrf(n, A, c_vp(ipiv), K, pivot, ctypes.byref(o) if o is not None else None,
                           c_vp(info) if info else None, c_vp(stream))


def dd_getrs(n, nrhs, LU: dd_mat, ipiv: int, B: dd_mat, stream: int = 0) -> int:
    return load().dd_getrs(n, nrhs, LU, c_vp(ipiv), B, c_vp(stream))


DDG_BATCH_ONE_LEAF_LAUNCH = 1


def ddg_batch_create(problems, use_graph: bool = False, stream: int = 0, flags: int = 0) -> int:
    arr = (ddg_problem * max(len(problems), 1))(*problems)
    h = c_vp()
    check(load().ddg_batch_create_ex(ctypes.byref(h), len(problems), arr, 1 if use_graph else 0, flags,
                                     c_vp(stream)))
    return h.value


def ddg_batch_run(handle: int, stream: int = 0) -> None:
    check(load().ddg_batch_run(c_vp(handle), c_vp(stream)))


def ddg_batch_get_stats(handle: int) -> dict:
    st = ddg_batch_stats()
    check(load().ddg_batch_get_stats(c_vp(handle), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in ddg_batch_stats._fields_}


def ddg_batch_destroy(handle: int, stream: int = 0) -> None:
    check(load().ddg_batch_destroy(c_vp(handle), c_vp(stream)))


def dd_gemm_batched(problems, stream: int = 0) -> int:
    arr = (ddg_problem * max(len(problems), 1))(*problems)
    return load().dd_gemm_batched(len(problems), arr, c_vp(stream))


def qd_getrf(n, A: qd_mat, ipiv: int, K: int, pivot: int, o: ddg_opts | None, info: int | None,
             stream: int = 0) -> int:
    return load().qd_getrf(n, A, c_vp(ipiv), K, pivot, ctypes.byref(o) if o is not None else None,
                           c_vp(info) if info else None, c_vp(stream))


def qd_getrs(n, nrhs, LU: qd_mat, ipiv: int, B: qd_mat, stream: int = 0) -> int:
    return load().qd_getrs(n, nrhs, LU, c_vp(ipiv), B, c_vp(stream))


def ddg_workspace_reserve(device: int, nbytes: int) -> None:
    check(load().ddg_workspace_reserve(device, nbytes))


def ddg_workspace_release(device: int) -> None:
    check(load().ddg_workspace_release(device))


def ddg_workspace_stats(device: int) -> dict:
    st = ddg_workspace_info()
    check(load().ddg_workspace_stats(device, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in ddg_workspace_info._fields_}
