"""Communication lower bounds and processor grids of arXiv 2603.20966.

Host-side utility (no GPU work): the words a load-balanced parallel algorithm
with P processors must move for

* B = A Omega with A n1 x n2 and a random Omega n2 x r, n2 > r
  (Sec. 3, Theorem 2 "randMatmulLB"), together with the grid
  p1 x p2 x p3 of the paper's algorithm (Sec. 3.3, Cases 1-3) and that
  algorithm's bandwidth and latency costs (Sec. 3.2 cost analysis);
* the Nystrom pair B = A Omega, C = Omega^T B with A n x n symmetric and
  Omega n x r, n > r (Sec. 5, Theorem "NystromLB").

The transposed product C^T = Omega^T A^T has the same bound (the remark after
Theorem 2), which is the left sketch of this library.  On one GPU every
sketch is Case 1 (P = 1 <= n1): no communication.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


def randmatmul_lower_bound(n1: float, n2: float, r: float, P: float) -> float:
    """Theorem 2: words moved by some processor, at least."""
    if P <= n1:
        return 0.0
    if P <= n1 * n2 / r:
        return r - n1 * r / P
    return 2.0 * math.sqrt(n1 * n2 * r / P) - (n1 * n2 + n1 * r) / P


@dataclass(frozen=True)
class Grid:
    p1: float
    p2: float
    p3: float
    case: int


def randmatmul_grid(n1: float, n2: float, r: float, P: float) -> Grid:
    """The processor grid of Sec. 3.3 for each case of Theorem 2 (real-valued:
    the paper assumes the divisions are exact)."""
    if P <= n1:
        return Grid(P, 1.0, 1.0, 1)
    if P <= n1 * n2 / r:
        return Grid(n1, P / n1, 1.0, 2)
    return Grid(n1, math.sqrt(P * n2 / (r * n1)), math.sqrt(P * r / (n1 * n2)), 3)


def randmatmul_cost(n1: float, n2: float, r: float, g: Grid) -> tuple[float, float]:
    """(bandwidth, latency) of the paper's Alg. 1 on grid g: an All-Gather of
    A blocks over p3 processors and a Reduce-Scatter of B blocks over p2."""
    P = g.p1 * g.p2 * g.p3
    bw = n1 * n2 / (g.p1 * g.p2) + n1 * r / (g.p1 * g.p3) - (n1 * n2 + n1 * r) / P
    lat = math.log2(g.p3) + math.log2(g.p2)
    return bw, lat


def gemm_lower_bound(n1: float, n2: float, r: float, P: float) -> float:
    """The general matrix-multiplication bound the paper compares with
    (n1 >= n2 > r), the three regimes drawn after Theorem 2."""
    if P <= n1 / n2:
        return n2 * r - n2 * r / P
    if P <= n1 * n2 / (r * r):
        return 2.0 * math.sqrt(n1 * n2 * r * r / P) - (n1 * r + n2 * r) / P
    return 3.0 * (n1 * n2 * r / P) ** (2.0 / 3.0) - (n1 * r + n2 * r + n1 * n2) / P


def nystrom_accessed(n: float, r: float, P: float) -> float:
    """W of the Nystrom theorem: the fewest elements of A, B, C one processor
    must access."""
    if P <= r:
        return (n * n + n * r + r * r) / P
    if P <= n:
        return (n * n + n * r) / P + r
    if P <= n * (n + r) / r:
        return n * n / P + r + n * r / P
    return 2.0 * math.sqrt(n * r * (n + r) / P)


def nystrom_lower_bound(n: float, r: float, P: float) -> float:
    """Nystrom theorem: words moved, at least W - (n^2 + nr + r^2)/P."""
    return nystrom_accessed(n, r, P) - (n * n + n * r + r * r) / P
