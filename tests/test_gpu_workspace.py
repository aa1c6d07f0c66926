"""The library's workspace pool (ddg_workspace_reserve / release / stats):
a reservation keeps the pool mapped between calls and leaves results
bit-identical; release returns the unused memory; a reservation that cannot
be had is DDG_ENOMEM and holds nothing."""
import pytest

from paper_1510_08642_gb300 import inputs as I
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1510_08642_gb300 as P
    P.capi.load()


def test_reserve_keeps_memory_and_results():
    import paper_1510_08642_gb300 as P
    cap = P.capi
    dev = torch.cuda.current_device()
    n = 1024
    A = to_dev(I.uniform(n, n, 2, seed=11))
    B = to_dev(I.uniform(n, n, 2, seed=12))
    C0 = P.gemm(A, B, algo="winograd", cutoff=256)
    torch.cuda.synchronize()
    st = cap.ddg_workspace_stats(dev)
    assert st["used_high_bytes"] > 0        # the recursion's temporaries came from the pool
    assert st["used_bytes"] == 0
    cap.ddg_workspace_reserve(dev, 512 * MiB)
    st = cap.ddg_workspace_stats(dev)
    assert st["threshold_bytes"] == 512 * MiB
    assert st["reserved_bytes"] >= 512 * MiB
    C1 = P.gemm(A, B, algo="winograd", cutoff=256)
    torch.cuda.synchronize()
    st = cap.ddg_workspace_stats(dev)
    assert st["reserved_bytes"] >= 512 * MiB  # still mapped after the synchronisation
    assert st["used_bytes"] == 0
    assert torch.equal(C0, C1)
    cap.ddg_workspace_release(dev)
    torch.cuda.synchronize()
    st = cap.ddg_workspace_stats(dev)
    assert st["threshold_bytes"] == 0
    assert st["reserved_bytes"] < 512 * MiB


def test_reserve_too_much_is_enomem():
    import paper_1510_08642_gb300 as P
    cap = P.capi
    dev = torch.cuda.current_device()
    st = cap.load().ddg_workspace_reserve(dev, 1 << 52)   # 4 PiB: never available
    assert st == cap.DDG_ENOMEM, cap.last_error()
    assert cap.ddg_workspace_stats(dev)["threshold_bytes"] == 0
    # the library still works afterwards
    A = to_dev(I.uniform(64, 64, 2, seed=1))
    C = P.gemm(A, A, algo="block")
    torch.cuda.synchronize()
    assert torch.isfinite(C).all()


def test_bad_device_is_einval():
    import paper_1510_08642_gb300 as P
    cap = P.capi
    assert cap.load().ddg_workspace_reserve(torch.cuda.device_count(), MiB) == cap.DDG_EINVAL
