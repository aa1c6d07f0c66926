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
