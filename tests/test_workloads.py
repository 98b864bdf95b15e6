"""Input recipes of the benchmark workloads (host only)."""
import math

import pytest

from paper_2603_20966_gb300.workloads import batched_problems, serving_requests


def test_batched_problems_ranges():
    ps = batched_problems(256, seed=1000)
    assert len(ps) == 256
    assert all(1024 <= p.m <= 65536 and 32 <= p.n <= 512 and p.k == 2 * p.n for p in ps)
    assert {p.dist for p in ps} == {0, 1}
    assert [p.seed for p in ps] == list(range(1000, 1256))


def test_serving_stream_shape():
    rs = serving_requests(20000, rate=2000.0, seed=3000)
    assert len(rs) == 20000
    arr = [r.arrival_s for r in rs]
    assert arr[0] == 0.0 and all(b >= a for a, b in zip(arr, arr[1:]))
    # Poisson process: mean gap 1/rate within a few standard errors
    mean_gap = arr[-1] / (len(rs) - 1)
    assert abs(mean_gap - 5e-4) < 4 * 5e-4 / math.sqrt(len(rs))
    assert all(1024 <= r.prob.m <= 1 << 18 for r in rs)
    assert all(0 <= r.row0 and r.row0 + r.prob.m <= 1 << 18 for r in rs)
    # log-uniform m: the median is the geometric mean of the ends
    ms = sorted(r.prob.m for r in rs)
    assert ms[len(ms) // 2] == pytest.approx(math.sqrt(1024 * (1 << 18)), rel=0.05)
