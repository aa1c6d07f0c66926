"""The continuous-batching server on the GPU: every result is the same alone
and in the mix (bit-identical: same kernels and order), a small memory
budget still completes, and the latency statistics are filled in."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def small_requests(count, rate, seed):
    from paper_1510_08642_gb300 import serving as S
    return S.poisson_requests(count, rate, seed, gemm_n=(40, 300), lu_n=(64, 130, 257))


def test_results_same_alone_and_in_mix():
    from paper_1510_08642_gb300 import serving as S
    srv = S.Server(slots=3, keep_results=True, gemm_cutoff=64, lu_K=32, lu_cutoff=16, max_batch=8)
    mix = small_requests(30, 400.0, seed=5)
    st = srv.run(mix)
    assert st["all"]["count"] == 30
    assert st["gemm"]["p99_ms"] >= st["gemm"]["p50_ms"] > 0
    for r in mix:
        alone = S.Request(r.rid, r.kind, r.n, 0.0, r.seed)
        srv.run([alone])
        a, b = r.result.cpu().numpy(), alone.result.cpu().numpy()
        assert np.array_equal(a, b), (r.kind, r.n)
        assert r.info == 0
        if r.kind == "lu":  # solution of A x = A 1
            assert np.abs(a[0] - 1.0 + a[1]).max() < 1e-20
    srv.close()


def test_small_budget_serialises_but_completes():
    from paper_1510_08642_gb300 import serving as S
    srv = S.Server(slots=4, hbm_budget=1 << 20, gemm_cutoff=64, lu_K=32, lu_cutoff=16)
    reqs = small_requests(12, 0.0, seed=6)
    st = srv.run(reqs)
    assert st["all"]["count"] == 12
    assert all(np.isfinite(r.done) and r.done >= r.arrival for r in reqs)
    srv.close()
