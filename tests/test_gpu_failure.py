"""Failure detection on the GPU without a fault: the library's bounded
device waits give up, the kernel returns and the host reads the status.

Each test runs a wait on a barrier that nothing completes (the tensor-core
kernel with its TMA producer idle; an LU panel whose grid barrier expects
one arrival more than there are CTAs), checks the reported status, and then
checks that the context is still usable: a normal product or factorisation
right after gives correct results and no further timeouts."""
import numpy as np
import pytest

import oracle as O
from paper_1510_08642_gb300 import inputs as I
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tensor_core_wait_runs_out_and_context_survives():
    import oracle.ozaki as OZ
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    capi.ddg_device_timeouts(reset=True)
    assert capi.ddg_test_bounded_wait(0) == capi.DDG_ETIMEOUT
    assert "as intended" in capi.last_error()
    assert capi.ddg_device_timeouts(reset=True) >= 1
    A = I.uniform(130, 200, 2, seed=400)
    B = I.uniform(200, 140, 2, seed=401)
    C = to_host(P.gemm(to_dev(A), to_dev(B), algo="ozaki2_tc", slices=32))
    want, _ = OZ.gemm_crt(A, B, 32)
    assert np.array_equal(C.view(np.uint64), want.view(np.uint64))
    assert capi.ddg_device_timeouts() == 0


def test_lu_panel_wait_runs_out_and_context_survives():
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    assert capi.ddg_test_bounded_wait(1) == capi.DDG_ETIMEOUT
    assert "panel barrier" in capi.last_error()
    n = 200
    A = I.uniform(n, n, 2, seed=402)
    dA = to_dev(A)
    ipiv = P.getrf(dA, K=64, pivot=True, algo="winograd", cutoff=32)
    torch.cuda.synchronize()
    _, piv_o, info = O.dd_getrf(A, pivot=True)
    assert info == 0 and np.array_equal(ipiv.cpu().numpy(), piv_o)


def test_bounded_wait_rejects_unknown_case():
    from paper_1510_08642_gb300 import capi
    assert capi.ddg_test_bounded_wait(7) == capi.DDG_EINVAL
