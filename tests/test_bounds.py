"""Pins of the communication-bound utility (host only): continuity at every
case boundary, the paper's algorithm attaining Theorem 2 on its chosen grid,
the bound never above the general GEMM bound (for every P with work to
balance), and the Nystrom bound's boundaries and limits."""
import math

import pytest

from paper_2603_20966_gb300 import bounds as B

SHAPES = [(1e6, 1e6, 1e3), (2 ** 20, 512, 64), (5e4, 5e4, 500), (4096, 2048, 16)]


@pytest.mark.parametrize("n1,n2,r", SHAPES)
def test_randmatmul_continuous_at_case_boundaries(n1, n2, r):
    for P in (n1, n1 * n2 / r):
        lo, hi = B.randmatmul_lower_bound(n1, n2, r, P * (1 - 1e-12)), \
            B.randmatmul_lower_bound(n1, n2, r, P * (1 + 1e-12))
        assert lo == pytest.approx(hi, rel=1e-6, abs=1e-6)
    # closed forms at the two boundaries
    assert B.randmatmul_lower_bound(n1, n2, r, n1) == 0.0
    assert B.randmatmul_lower_bound(n1, n2, r, n1 * n2 / r) == pytest.approx(r - r * r / n2)


@pytest.mark.parametrize("n1,n2,r", SHAPES)
def test_algorithm_attains_the_bound(n1, n2, r):
    # Sec. 3.3: the grid of each case makes Alg. 1's bandwidth equal the bound
    for P in (1, n1 / 2, n1, 3 * n1, n1 * n2 / r, 10 * n1 * n2 / r, 1e3 * n1 * n2 / r):
        g = B.randmatmul_grid(n1, n2, r, P)
        assert g.p1 * g.p2 * g.p3 == pytest.approx(P, rel=1e-12)
        bw, lat = B.randmatmul_cost(n1, n2, r, g)
        lb = B.randmatmul_lower_bound(n1, n2, r, P)
        assert bw == pytest.approx(lb, rel=1e-9, abs=1e-6 * max(1.0, abs(lb)))
        if g.case == 1:
            assert bw == pytest.approx(0.0, abs=1e-6) and lat == 0.0


@pytest.mark.parametrize("n1,n2,r", [s for s in SHAPES if s[0] >= s[1]])
def test_not_above_gemm_bound(n1, n2, r):
    # over every processor count that still has work to balance (P <= n1 n2 r)
    for e in range(0, int(math.log2(n1 * n2 * r)) + 1):
        P = 2.0 ** e
        assert B.randmatmul_lower_bound(n1, n2, r, P) <= B.gemm_lower_bound(n1, n2, r, P) + 1e-6


def test_randmatmul_case_examples():
    # one GPU, or as many processors as rows: nothing to move
    assert B.randmatmul_lower_bound(2 ** 20, 512, 2048, 1) == 0.0
    g = B.randmatmul_grid(2 ** 20, 512, 2048, 8)
    assert (g.p1, g.p2, g.p3, g.case) == (8, 1, 1, 1)
    # case 3 grid dimensions
    g = B.randmatmul_grid(100, 100, 10, 4000)
    assert g.case == 3 and g.p2 == pytest.approx(20.0) and g.p3 == pytest.approx(2.0)


@pytest.mark.parametrize("n,r", [(5e4, 500), (1e6, 1e3), (4096, 64)])
def test_nystrom_boundaries_and_limits(n, r):
    for P in (r, n, n * (n + r) / r):
        lo = B.nystrom_accessed(n, r, P * (1 - 1e-12))
        hi = B.nystrom_accessed(n, r, P * (1 + 1e-12))
        assert lo == pytest.approx(hi, rel=1e-6)
    # one processor owns everything: nothing to move
    assert B.nystrom_lower_bound(n, r, 1) == pytest.approx(0.0, abs=1e-6)
    # at the last boundary the accessed volume is exactly 2r
    assert B.nystrom_accessed(n, r, n * (n + r) / r) == pytest.approx(2 * r)
    # never negative, never more than all the data
    for e in range(0, int(math.log2(n * n * r)) + 1):
        w = B.nystrom_lower_bound(n, r, 2.0 ** e)
        assert -1e-6 <= w <= n * n + n * r + r * r


def test_nystrom_at_least_each_product():
    # the pair moves at least what its first product alone must move
    n, r = 5e4, 500
    for e in range(0, int(math.log2(n * n * r)) + 1):
        P = 2.0 ** e
        assert B.nystrom_lower_bound(n, r, P) >= B.randmatmul_lower_bound(n, n, r, P) - 1e-6
