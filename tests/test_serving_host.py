"""Serving loop host logic: the request generator and the footprint model."""
import numpy as np

from paper_1510_08642_gb300 import serving as S


def test_poisson_requests_deterministic_mix():
    a = S.poisson_requests(400, 5.0, seed=3)
    b = S.poisson_requests(400, 5.0, seed=3)
    assert [(r.kind, r.n, r.arrival) for r in a] == [(r.kind, r.n, r.arrival) for r in b]
    kinds = [r.kind for r in a]
    assert 0.4 < kinds.count("gemm") / len(kinds) < 0.6
    g = [r.n for r in a if r.kind == "gemm"]
    assert min(g) >= 256 and max(g) <= 2048
    assert set(r.n for r in a if r.kind == "lu") <= {1024, 2048, 4096}
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) >= 0) and t[0] == 0.0
    # mean gap ~ 1 / rate
    assert 0.15 < np.diff(t).mean() < 0.25


def test_saturation_requests_arrive_together():
    a = S.poisson_requests(10, 0.0, seed=1)
    assert all(r.arrival == 0.0 for r in a)


def test_footprint_grows_with_n():
    small = S.Request(0, "gemm", 256, 0.0, 1)
    big = S.Request(1, "gemm", 2048, 0.0, 1)
    lu = S.Request(2, "lu", 4096, 0.0, 1)
    assert S.footprint(small) < S.footprint(big)
    assert S.footprint(lu) >= 2 * 4096 * 4096 * 16


def test_stats_percentiles():
    rs = [S.Request(i, "gemm", 256, 0.0, i) for i in range(100)]
    for i, r in enumerate(rs):
        r.done = (i + 1) * 1e-3
    st = S.stats(rs)
    assert abs(st["gemm"]["p50_ms"] - 50.5) < 1e-6
    assert st["gemm"]["p99_ms"] > 99.0


def test_check_request_refusals():
    ok = S.Request(0, "gemm", 512, 0.0, 1)
    assert S.check_request(ok, 1 << 40, 16384) == ""
    assert "kind" in S.check_request(S.Request(1, "qr", 512, 0.0, 1), 1 << 40, 16384)
    assert "positive" in S.check_request(S.Request(2, "lu", 0, 0.0, 1), 1 << 40, 16384)
    assert "positive" in S.check_request(S.Request(3, "lu", 2.5, 0.0, 1), 1 << 40, 16384)
    assert "limit" in S.check_request(S.Request(4, "lu", 20000, 0.0, 1), 1 << 40, 16384)
    big = S.Request(5, "gemm", 4096, 0.0, 1)
    assert "budget" in S.check_request(big, S.footprint(big) - 1, 16384)
    assert S.check_request(big, S.footprint(big), 16384) == ""


def test_admission_deadline():
    r = S.Request(0, "gemm", 256, 1.0, 1, deadline=0.5)
    assert not S.expired(r, 1.2) and not S.expired(r, 1.5)
    assert S.expired(r, 1.5001)
    assert not S.expired(S.Request(1, "lu", 1024, 0.0, 1), 1e9)  # no deadline


def test_stats_count_refusals_apart():
    rs = [S.Request(i, "gemm", 256, 0.0, i) for i in range(10)]
    for i, r in enumerate(rs):
        r.done, r.status = (i + 1) * 1e-3, "ok"
    rs[0].status, rs[1].status = "refused", "timeout"
    st = S.stats(rs)
    assert st["gemm"]["count"] == 8 and st["refused"] == 1 and st["timeout"] == 1
