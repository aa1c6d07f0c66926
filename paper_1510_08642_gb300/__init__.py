"""DD / QD matrix products and LU on one GB300 (Kouya 2015, GB300-native).

The compute path is the CUDA library libddgemm.so (C ABI: include/ddgemm.h).
This package holds its build script (build.py), the ctypes binding
(capi.py), thin torch helpers below that pass device pointers of torch
tensors through the C ABI, and the seeded input generator (inputs.py).

A DD matrix is a float64 tensor of shape (2, rows, cols) (planes hi, lo), a
QD matrix one of shape (4, rows, cols); planes must be row-contiguous.
"""
from __future__ import annotations

from . import capi


def _mat(T, limbs: int):
    """The C-ABI view (planes and leading dimension) of a DD / QD tensor of
    shape (limbs, rows, cols): float64 on a CUDA device, each row contiguous,
    rows not overlapping. Raises TypeError / ValueError otherwise, so that
    the library never sees a layout that would take it outside the tensor."""
    import torch
    if not isinstance(T, torch.Tensor) or T.dtype != torch.float64:
        raise TypeError(f"float64 tensor expected, got {getattr(T, 'dtype', type(T))}")
    if T.dim() != 3 or T.shape[0] != limbs:
        raise ValueError(f"expected shape ({limbs}, rows, cols), got {tuple(T.shape)}")
    rows, cols = T.shape[1], T.shape[2]
    empty = rows == 0 or cols == 0
    if not empty and cols > 1 and T.stride(2) != 1:
        raise ValueError("each row must be contiguous (stride 1 along the last dimension)")
    if not empty and rows > 1 and T.stride(1) < cols:
        raise ValueError(f"rows overlap (row stride {T.stride(1)} < {cols} columns)")
    if not T.is_cuda:
        raise ValueError("CUDA tensor expected")
    ld = max(T.stride(1), cols) if not empty else max(cols, 1)
    ps = T.stride(0)
    base = T.data_ptr()
    ptrs = [base + q * ps * 8 for q in range(limbs)]
    if limbs == 2:
        return capi.dd_mat(ptrs[0], ptrs[1], max(ld, 1))
    m = capi.qd_mat()
    for q in range(4):
        m.x[q] = ptrs[q]
    m.ld = max(ld, 1)
    return m


def gemm(A, B, C=None, algo: str = "winograd", cutoff: int = 512, mode: str = "set",
         pad: bool = False, streams: int = 7, accum: str = "fx", slices: int = 0, stream=None):
    """C (mode) A B through dd_gemm / qd_gemm on the current CUDA stream.

    A: (limbs, m, l), B: (limbs, l, n), C: (limbs, m, n) or None (allocated).
    limbs = 2 (DD) or 4 (QD). accum: "fx" (fixed-point window, default),
    "fx_tile" (the same bits, tiles converted as they are staged, no operand
    workspace) or "twosum" for the Block base case. Returns C.
    """
    import torch

    if A.dim() != 3 or B.dim() != 3 or A.shape[0] not in (2, 4):
        raise ValueError(f"A and B must be (2 or 4, rows, cols) tensors, got {tuple(A.shape)}, {tuple(B.shape)}")
    limbs, m, l = A.shape
    if B.shape[0] != limbs or B.shape[1] != l:
        raise ValueError(f"B must be ({limbs}, {l}, n) for A of shape {tuple(A.shape)}, got {tuple(B.shape)}")
    n = B.shape[2]
    if C is None:
        C = torch.empty((limbs, m, n), dtype=torch.float64, device=A.device)
    elif tuple(C.shape) != (limbs, m, n):
        raise ValueError(f"C must be {(limbs, m, n)}, got {tuple(C.shape)}")
    o = capi.opts(algo, cutoff, pad, streams, accum, slices)
    s = (stream or torch.cuda.current_stream(A.device)).cuda_stream
    fn = capi.dd_gemm if limbs == 2 else capi.qd_gemm
    capi.check(fn(m, l, n, _mat(A, limbs), _mat(B, limbs), _mat(C, limbs), capi.MODES[mode], o, s))
    return C


def getrf(A, K: int = 64, pivot: bool = True, algo: str = "winograd", cutoff: int = 32,
          accum: str = "fx", info=None, stream=None):
    """In-place DD / QD LU through dd_getrf / qd_getrf (by A's limb count);
    returns the device ipiv (int64, n)."""
    import torch

    if A.dim() != 3 or A.shape[0] not in (2, 4) or A.shape[1] != A.shape[2]:
        raise ValueError(f"a square (2 or 4, n, n) matrix expected, got {tuple(A.shape)}")
    if info is not None and (info.dtype != torch.int64 or info.numel() < 1 or not info.is_cuda):
        raise ValueError("info must be an int64 CUDA tensor of at least one element")
    limbs, n = A.shape[0], A.shape[1]
    ipiv = torch.empty(n, dtype=torch.int64, device=A.device)
    o = capi.opts(algo, cutoff, False, 7, accum)
    s = (stream or torch.cuda.current_stream(A.device)).cuda_stream
    fn = capi.dd_getrf if limbs == 2 else capi.qd_getrf
    capi.check(fn(n, _mat(A, limbs), ipiv.data_ptr(), K, 1 if pivot else 0, o,
                  info.data_ptr() if info is not None else None, s))
    return ipiv


def getrs(LU, ipiv, B, stream=None):
    """Solve with dd_getrs / qd_getrs; B (limbs, n, nrhs) is overwritten with X."""
    import torch

    if LU.dim() != 3 or LU.shape[0] not in (2, 4) or LU.shape[1] != LU.shape[2]:
        raise ValueError(f"a square (2 or 4, n, n) factor expected, got {tuple(LU.shape)}")
    if B.dim() != 3 or B.shape[0] != LU.shape[0] or B.shape[1] != LU.shape[1]:
        raise ValueError(f"B must be {(LU.shape[0], LU.shape[1])} x nrhs, got {tuple(B.shape)}")
    limbs, n, nrhs = B.shape
    if (ipiv.dtype != torch.int64 or ipiv.dim() != 1 or ipiv.numel() < n or not ipiv.is_cuda
            or not ipiv.is_contiguous()):
        raise ValueError(f"ipiv must be a contiguous int64 CUDA tensor of {n} entries")
    s = (stream or torch.cuda.current_stream(LU.device)).cuda_stream
    fn = capi.dd_getrs if limbs == 2 else capi.qd_getrs
    capi.check(fn(n, nrhs, _mat(LU, limbs), ipiv.data_ptr(), _mat(B, limbs), s))
    return B


def problem(A, B, C, algo: str = "block", cutoff: int = 512, mode: str = "set"):
    """A ddg_problem for the batched entry points from three device tensors."""
    if A.dim() != 3 or B.dim() != 3 or C.dim() != 3 or A.shape[0] not in (2, 4):
        raise ValueError("A, B and C must be (2 or 4, rows, cols) tensors")
    limbs = A.shape[0]
    if B.shape[0] != limbs or B.shape[1] != A.shape[2] or tuple(C.shape) != (limbs, A.shape[1], B.shape[2]):
        raise ValueError(f"shapes {tuple(A.shape)} x {tuple(B.shape)} -> {tuple(C.shape)} do not agree")
    p = capi.ddg_problem()
    p.limbs = limbs
    p.mode = capi.MODES[mode]
    p.m, p.l, p.n = A.shape[1], A.shape[2], B.shape[2]
    for name, T in (("A", A), ("B", B), ("C", C)):
        mt = _mat(T, limbs)
        ptrs = [mt.hi, mt.lo] if limbs == 2 else list(mt.x)
        arr = getattr(p, name)
        for q in range(limbs):
            arr[q] = ptrs[q]
        setattr(p, "ld" + name.lower(), mt.ld)
    p.algo = capi.ALGOS[algo]
    p.cutoff = cutoff
    p._tensors = (A, B, C)  # a plan made from p keeps them alive (Batch holds its problems)
    return p


class Batch:
    """A batch plan (ddg_batch): grouped launches, optionally a CUDA graph.
    The plan addresses the problems' matrices by pointer; it holds the
    problems made by `problem`, and with them their tensors, so that none is
    freed while the plan can still run."""

    def __init__(self, problems, use_graph: bool = False, stream=None, one_launch: bool = False):
        """one_launch: every base-case product (DD and QD) in one persistent
        grouped launch, tiles converted as staged (DDG_BATCH_ONE_LEAF_LAUNCH;
        the same bits)."""
        import torch
        self.problems = list(problems)
        self.stream = stream or torch.cuda.current_stream()
        self.handle = capi.ddg_batch_create(self.problems, use_graph, self.stream.cuda_stream,
                                            capi.DDG_BATCH_ONE_LEAF_LAUNCH if one_launch else 0)
        self.stats = capi.ddg_batch_get_stats(self.handle)

    def run(self, stream=None):
        capi.ddg_batch_run(self.handle, (stream or self.stream).cuda_stream)

    def close(self, stream=None):
        if self.handle:
            capi.ddg_batch_destroy(self.handle, (stream or self.stream).cuda_stream)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
