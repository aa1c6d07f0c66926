"""The continuous-batching server on the GPU.

* Every served result is checked against the CPU oracle: each GEMM's exact
  error (Kulisch checker) within the normwise bound of its algorithm, each
  LU solve's exact residual ||b - A x|| / (||A|| ||x||) <= n 2^-100
  (Section 4, Eq. 2), on the operands the server generated on the device.
* Every result is the same alone and in the mix (bit-identical: same
  kernels and order).
* A small memory budget still completes; malformed, oversized and expired
  requests are refused or cancelled without disturbing the others (faults
  injected on the host: no GPU fault, trap or hang).
"""
import numpy as np
import pytest

import oracle as O
from tests.gpu_util import normwise_bound

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def small_requests(count, rate, seed):
    from paper_1510_08642_gb300 import serving as S
    return S.poisson_requests(count, rate, seed, gemm_n=(40, 300), lu_n=(64, 130, 257))


def check_against_oracle(r, gemm_cutoff):
    """The result of served request r against the oracle (r.operands kept)."""
    if r.kind == "gemm":
        A, B = (t.cpu().numpy() for t in r.operands)
        C = r.result.cpu().numpy()
        err = O.gemm_error(A, B, C)
        algo = "winograd" if r.n > gemm_cutoff else "block"
        assert O.normwise(err, A, B) <= normwise_bound(r.n, 2, algo), (r.rid, r.n)
    else:
        A, b = (t.cpu().numpy() for t in r.operands)
        x = r.result.cpu().numpy()
        res = O.dd_residual(A, x, b)
        rel = np.abs(res).max() / (np.abs(A[0]).sum(axis=1).max() * np.abs(x[0]).max())
        assert rel <= r.n * 2.0 ** -100, (r.rid, r.n, rel)
        assert np.abs(x[0] - 1.0 + x[1]).max() < 1e-20  # b = A 1, cond(A) ~ 1e4-1e6


def test_results_match_oracle_and_same_alone_and_in_mix():
    from paper_1510_08642_gb300 import serving as S
    srv = S.Server(slots=3, keep_results=True, gemm_cutoff=64, lu_K=32, lu_cutoff=16, max_batch=8)
    mix = small_requests(30, 400.0, seed=5)
    st = srv.run(mix)
    assert st["all"]["count"] == 30 and st["refused"] == 0 and st["timeout"] == 0
    assert st["gemm"]["p99_ms"] >= st["gemm"]["p50_ms"] > 0
    assert {r.kind for r in mix} == {"gemm", "lu"}
    for r in mix:
        assert r.status == "ok" and r.info == 0
        check_against_oracle(r, 64)
        alone = S.Request(r.rid, r.kind, r.n, 0.0, r.seed)
        srv.run([alone])
        a, b = r.result.cpu().numpy(), alone.result.cpu().numpy()
        assert np.array_equal(a, b), (r.kind, r.n)
    srv.close()


def test_small_budget_serialises_but_completes():
    from paper_1510_08642_gb300 import serving as S
    srv = S.Server(slots=4, hbm_budget=1 << 20, gemm_cutoff=64, lu_K=32, lu_cutoff=16)
    reqs = small_requests(12, 0.0, seed=6)
    for r in reqs:  # every request alone exceeds the budget: admitted one at a time
        r.n = min(r.n, 60)
    st = srv.run(reqs)
    assert st["all"]["count"] == 12
    assert all(r.status == "ok" and np.isfinite(r.done) and r.done >= r.arrival for r in reqs)
    srv.close()


def test_refused_and_expired_requests_leave_the_rest_correct():
    """Host-injected faults: a malformed kind, a zero order, an order above
    the server's limit, a footprint above the budget and an admission
    deadline that has already passed. Those end refused / timed out with a
    reason and launch nothing; the others are served and match the oracle."""
    from paper_1510_08642_gb300 import serving as S
    from paper_1510_08642_gb300 import capi
    srv = S.Server(slots=3, keep_results=True, gemm_cutoff=64, lu_K=32, lu_cutoff=16, max_batch=8,
                   hbm_budget=64 << 20, max_n=1024)
    good = small_requests(8, 0.0, seed=7)
    bad = [S.Request(100, "svd", 64, 0.0, 1), S.Request(101, "gemm", 0, 0.0, 1),
           S.Request(102, "lu", 2048, 0.0, 1), S.Request(103, "gemm", 1000, 0.0, 1),
           S.Request(104, "gemm", 64, 0.0, 1, deadline=-1.0)]
    launches = capi.ddg_kernel_launches()
    st = srv.run(good + bad)
    assert st["refused"] == 4 and st["timeout"] == 1
    assert [r.status for r in bad] == ["refused"] * 4 + ["timeout"]
    assert "kind" in bad[0].error and "positive" in bad[1].error and "limit" in bad[2].error
    assert "budget" in bad[3].error and "admitted" in bad[4].error
    assert all(r.result is None for r in bad)
    assert st["all"]["count"] == len(good)
    for r in good:
        assert r.status == "ok"
        check_against_oracle(r, 64)
    # only the good requests launched work
    assert capi.ddg_kernel_launches() > launches
    srv.close()
