"""Host-side logic of the serving loop: arrivals, admission accounting, latency statistics
(CPU only)."""
import math

import numpy as np
import pytest

from paper_2508_04701_gb300 import serve


def test_poisson_arrivals_rate_and_determinism():
    a = serve.poisson_requests(rate=2000, duration=10.0, n_facts=512, seed=0)
    b = serve.poisson_requests(rate=2000, duration=10.0, n_facts=512, seed=0)
    assert [(r.arrival, r.fact_id, r.t) for r in a] == [(r.arrival, r.fact_id, r.t) for r in b]
    # count of a Poisson process over 10 s at 2000/s: 20 000 +- 3 sigma (sigma ~ 141)
    assert abs(len(a) - 20_000) < 450
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) >= 0) and arr[-1] <= 10.0
    gaps = np.diff(arr)
    assert abs(gaps.mean() - 1 / 2000) < 3 * (1 / 2000) / math.sqrt(gaps.size)
    # exponential gaps: coefficient of variation ~ 1
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05
    ts = np.array([r.t for r in a])
    assert ts.min() >= 5 and ts.max() <= 90
    facts = np.array([r.fact_id for r in a])
    assert facts.min() >= 0 and facts.max() < 512


def test_admission_accounting():
    adm = serve.Admission(budget_bytes=1000, resident_bytes=600)
    assert adm.fits(400) and not adm.fits(401)
    adm.take(300)
    assert adm.fits(100) and not adm.fits(101)
    adm.give(300)
    assert adm.in_flight == 0 and adm.fits(400)


def test_latency_stats():
    reqs = []
    for i in range(1000):
        r = serve.Request(i, 0, 50, arrival=i * 0.001)
        r.done = r.arrival + (0.002 if i % 100 else 0.050)
        reqs.append(r)
    st = serve.latency_stats(reqs)
    assert st["requests"] == 1000
    assert st["p50_ms"] == pytest.approx(2.0)
    assert st["max_ms"] == pytest.approx(50.0)
    assert 2.0 <= st["p99_ms"] <= 50.0
    assert st["throughput_qps"] == pytest.approx(1000 / (0.999 + 0.002), rel=1e-6)
    # warm-up requests are excluded
    assert serve.latency_stats(reqs, warmup=0.5)["requests"] == 500


def test_span_overlap_and_union():
    """Device-overlap bookkeeping of the serving loop: the most spans containing one instant,
    and the length their union covers (brute force over a fine grid)."""
    rng = np.random.default_rng(9)
    for _ in range(50):
        k = int(rng.integers(0, 8))
        a = rng.integers(0, 50, size=k)
        spans = [(float(x), float(x + rng.integers(1, 20))) for x in a]
        grid = np.arange(0, 80, 0.5) + 0.25
        cover = [sum(1 for s, e in spans if s <= g < e) for g in grid]
        assert serve.max_overlap(spans) == max(cover, default=0)
        assert serve.union_length(spans) == pytest.approx(0.5 * sum(1 for c in cover if c > 0))
    assert serve.max_overlap([(0.0, 1.0), (1.0, 2.0)]) == 1      # touching spans do not overlap
