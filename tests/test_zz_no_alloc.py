"""dd_gemm_noalloc: the product for callers that cannot allocate device memory.

Some callers of this library must not allocate at call time: services that
reserve their device memory once at start-up, host frameworks whose own
allocator already owns the free device memory, and latency-bound loops where
an allocation could stall or fail. dd_gemm_noalloc gives them the Strassen /
Winograd product with its temporaries in a fixed 64 MiB array compiled into
the library. These tests call it through the C ABI and check it against the
allocating entry point dd_gemm on two calls in a row (the second call sees
the first call's leftovers in the shared array), and check that an
oversized product is refused before anything is queued.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle as O
from paper_1510_08642_gb300 import inputs as I
from tests.gpu_util import normwise_bound, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _noalloc(dA, dB, dC, algo, cutoff, pad=False):
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    _, m, l = dA.shape
    n = dB.shape[2]
    o = capi.opts(algo, cutoff, pad, streams=1)
    s = torch.cuda.current_stream().cuda_stream
    st = capi.dd_gemm_noalloc(m, l, n, P._mat(dA, 2), P._mat(dB, 2), P._mat(dC, 2), capi.DDG_SET, o, s)
    capi.check(st)
    return dC


@pytest.mark.parametrize("algo,cutoff,shape,pad", [
    ("winograd", 64, (701, 513, 603), False),
    ("strassen", 48, (400, 384, 416), True),
])
def test_noalloc_matches_dd_gemm_two_calls(algo, cutoff, shape, pad):
    import paper_1510_08642_gb300 as P
    m, l, n = shape
    for call, seed in enumerate((40, 50)):
        A = I.uniform(m, l, 2, seed=seed)
        B = I.uniform(l, n, 2, seed=seed + 1)
        dA, dB = to_dev(A), to_dev(B)
        # the allocating entry point with the same algorithm, cutoff and
        # odd-size handling, its sub-products in order on one stream
        ref = P.gemm(dA, dB, algo=algo, cutoff=cutoff, pad=pad, streams=1)
        dC = torch.full((2, m, n), float("nan"), dtype=torch.float64, device="cuda")
        got = _noalloc(dA, dB, dC, algo, cutoff, pad)
        torch.cuda.synchronize()
        ref_h, got_h = to_host(ref), to_host(got)
        # the same arithmetic in the same order: the same bits, so stale
        # contents of the shared array (the first call's, on the second
        # call) cannot hide in a loose tolerance
        assert np.array_equal(ref_h.view(np.uint64), got_h.view(np.uint64)), call
        # and within the normwise bound of the other tests against the exact product
        err = O.gemm_error(A, B, got_h)
        assert O.normwise(err, A, B) <= normwise_bound(l, 2, algo)


def test_noalloc_refuses_oversized_product():
    """A product whose temporaries exceed the fixed array is refused before
    anything is queued: real operands (48 MiB), about 80 MiB of temporaries
    for a DD Winograd n = 1024 at cutoff 64, against the 64 MiB array."""
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    n = 1024
    dA = to_dev(I.uniform(n, n, 2, seed=60))
    dB = to_dev(I.uniform(n, n, 2, seed=61))
    dC = torch.zeros((2, n, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    launches = capi.ddg_kernel_launches()
    st = capi.dd_gemm_noalloc(n, n, n, P._mat(dA, 2), P._mat(dB, 2), P._mat(dC, 2), capi.DDG_SET,
                              capi.opts("winograd", 64, streams=1), torch.cuda.current_stream().cuda_stream)
    assert st == capi.DDG_EINVAL
    assert "fixed scratch" in capi.last_error()
    assert capi.ddg_kernel_launches() == launches
    torch.cuda.synchronize()
    assert not dC.any().item()
