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


def test_rbf_kernel_matrix_is_the_rbf_kernel():
    """The Nystrom workload's matrix: entries equal exp(-|x_i - x_j|^2 / (2 sigma^2))
    of the generated points with sigma^2 = |X|_F^2 / n (checked in FP64 against
    direct pairwise distances), so it is symmetric, has a unit diagonal and is
    positive semi-definite."""
    import numpy as np

    from paper_2603_20966_gb300.workloads import gaussian_matrix, rbf_kernel_matrix

    n, d = 700, 64
    K = rbf_kernel_matrix(n, d=d, seed=21, chunk_rows=256).double().numpy()
    X = gaussian_matrix(n, d, 21).double().numpy()
    sigma2 = (X * X).sum() / n
    D2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(axis=2)
    np.testing.assert_allclose(K, np.exp(-D2 / (2 * sigma2)), rtol=0, atol=2e-5)
    assert np.abs(K - K.T).max() <= 1e-6
    assert np.abs(np.diag(K) - 1.0).max() <= 1e-5
    assert np.linalg.eigvalsh(K).min() > -1e-4
