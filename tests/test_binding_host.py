"""The torch helpers' argument checks on the CPU: every layout or shape
that would let the library address memory outside a tensor is refused in
Python, before any pointer reaches the C ABI (CPU tensors stop at the
device check at the latest, so nothing here touches a GPU)."""
import pytest
import torch

import paper_1510_08642_gb300 as P


def z(*shape, dtype=torch.float64):
    return torch.zeros(shape, dtype=dtype)


def test_mat_refuses_layouts_outside_the_tensor():
    with pytest.raises(TypeError, match="float64"):
        P._mat(z(2, 4, 4, dtype=torch.float32), 2)
    with pytest.raises(TypeError, match="float64"):
        P._mat([[0.0]], 2)
    with pytest.raises(ValueError, match="shape"):
        P._mat(z(4, 4, 4), 2)
    with pytest.raises(ValueError, match="shape"):
        P._mat(z(2, 4), 2)
    with pytest.raises(ValueError, match="contiguous"):
        P._mat(z(2, 4, 6)[:, :, ::2], 2)
    with pytest.raises(ValueError, match="contiguous"):
        P._mat(z(2, 5, 4).transpose(1, 2), 2)
    # rows that overlap (a broadcast row): the library would read past the storage
    with pytest.raises(ValueError, match="rows overlap"):
        P._mat(z(2, 1, 5).expand(2, 4, 5), 2)
    # layouts the library can address: only the device is wrong
    for ok in (z(2, 4, 5), z(4, 3, 3), z(2, 0, 5), z(2, 3, 0), z(2, 1, 5).expand(2, 1, 5),
               z(2, 6, 4)[:, :, 1:2], z(2, 8, 8)[:, 2:6, 1:5]):
        with pytest.raises(ValueError, match="CUDA"):
            P._mat(ok, ok.shape[0])


def test_gemm_shapes_must_agree():
    A, B = z(2, 4, 5), z(2, 5, 3)
    with pytest.raises(ValueError, match="B must be"):
        P.gemm(A, z(2, 4, 3))
    with pytest.raises(ValueError, match="B must be"):
        P.gemm(A, z(4, 5, 3))
    with pytest.raises(ValueError, match="C must be"):
        P.gemm(A, B, z(2, 4, 4))
    with pytest.raises(ValueError, match="C must be"):
        P.gemm(A, B, z(4, 4, 3))
    with pytest.raises(ValueError, match="2 or 4"):
        P.gemm(z(3, 4, 5), z(3, 5, 3))
    with pytest.raises(ValueError, match="2 or 4"):
        P.gemm(z(4, 5), B)


def test_lu_shapes_and_index_arrays_checked():
    with pytest.raises(ValueError, match="square"):
        P.getrf(z(2, 4, 5))
    with pytest.raises(ValueError, match="square"):
        P.getrf(z(3, 4, 4))
    with pytest.raises(ValueError, match="info"):
        P.getrf(z(2, 4, 4), info=torch.zeros(1, dtype=torch.int32))
    with pytest.raises(ValueError, match="info"):
        P.getrf(z(2, 4, 4), info=torch.zeros(1, dtype=torch.int64))  # not on the device
    ipiv = torch.zeros(4, dtype=torch.int64)
    with pytest.raises(ValueError, match="square"):
        P.getrs(z(2, 4, 5), ipiv, z(2, 4, 1))
    with pytest.raises(ValueError, match="B must be"):
        P.getrs(z(2, 4, 4), ipiv, z(2, 5, 1))
    with pytest.raises(ValueError, match="B must be"):
        P.getrs(z(2, 4, 4), ipiv, z(4, 4, 1))
    for bad in (torch.zeros(3, dtype=torch.int64), torch.zeros(4, dtype=torch.int32),
                torch.zeros((4, 1), dtype=torch.int64), ipiv):  # short, narrow, 2-D, host memory
        with pytest.raises(ValueError, match="ipiv"):
            P.getrs(z(2, 4, 4), bad, z(2, 4, 2))


def test_batch_problem_shapes_must_agree():
    with pytest.raises(ValueError, match="do not agree"):
        P.problem(z(2, 4, 5), z(2, 4, 3), z(2, 4, 3))
    with pytest.raises(ValueError, match="do not agree"):
        P.problem(z(2, 4, 5), z(2, 5, 3), z(2, 4, 4))
    with pytest.raises(ValueError, match="do not agree"):
        P.problem(z(2, 4, 5), z(4, 5, 3), z(2, 4, 3))
    with pytest.raises(ValueError, match="2 or 4"):
        P.problem(z(2, 4, 5), z(2, 5, 3), z(4, 3))
    with pytest.raises(ValueError, match="CUDA"):  # consistent shapes reach the device check
        P.problem(z(2, 4, 5), z(2, 5, 3), z(2, 4, 3))


def test_batch_keeps_its_tensors_alive(monkeypatch):
    """A plan addresses its matrices by pointer: Batch holds the problems,
    and each problem its tensors, for as long as the plan exists (the
    device calls are replaced; only the references are checked)."""
    import gc
    import types
    import weakref
    from paper_1510_08642_gb300 import capi
    monkeypatch.setattr(P, "_mat", lambda T, limbs: capi.dd_mat(4096, 8192, max(T.shape[2], 1)))
    calls = []
    monkeypatch.setattr(capi, "ddg_batch_create", lambda probs, g, s, flags=0: calls.append(len(probs)) or 1)
    monkeypatch.setattr(capi, "ddg_batch_get_stats", lambda h: {"problems": calls[-1]})
    monkeypatch.setattr(capi, "ddg_batch_destroy", lambda h, s: None)
    stream = types.SimpleNamespace(cuda_stream=0)
    A, B, C = z(2, 4, 5), z(2, 5, 3), z(2, 4, 3)
    refs = [weakref.ref(t) for t in (A, B, C)]
    batch = P.Batch([P.problem(A, B, C)], stream=stream)
    del A, B, C
    gc.collect()
    assert all(r() is not None for r in refs) and batch.stats == {"problems": 1}
    batch.close()
    del batch
    gc.collect()
    assert all(r() is None for r in refs)
