"""Seeded synthetic inputs shaped like the sketching workloads.

This module holds no arithmetic of the sketch itself: it only draws the
dense input matrices A (with torch's own seeded generators) and describes
the benchmark configurations.  Tests hand the same tensors to the CUDA path
and to the CPU oracle.

Workloads (synthetic stand-ins for the paper's metabarcoding and CIFAR-10
kernel matrices, which are not available):
  C1  left,  A 4096 x 256 ~ N(0,1), k = 64, Gaussian (seed 7)
  C2  left,  A 2^20 x 512 ~ N(0,1), k = 2048, Rademacher and Gaussian
  C3  right, A = U V^T + 1e-3 E, U 65536 x 64, V 16384 x 64, E 65536 x 16384,
      all N(0,1); Omega 16384 x 256 Gaussian
  C4  256 independent left sketches, m log-uniform in [1024, 65536],
      n uniform in [32, 512], k = 2n, alternating distributions
  C5  Poisson stream of requests drawn like C4 with m up to 2^18
  NYS the Nystrom pair B = A Omega, C = Omega^T B of a 50000 x 50000 RBF
      kernel matrix (the shape of the paper's CIFAR-10 experiments), r = 500
      and 5000
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

A_SEED = 1
S_SEED = 7


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def gaussian_matrix(m: int, n: int, seed: int = A_SEED, device="cpu",
                    chunk_rows: int = 1 << 16) -> torch.Tensor:
    """A[m x n] with i.i.d. N(0,1) FP32 entries, drawn in row chunks so that
    very large matrices never need a second full-size temporary."""
    out = torch.empty((m, n), dtype=torch.float32, device=device)
    g = _gen(device, seed)
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        out[r0:r1].normal_(generator=g)
    return out


def lowrank_plus_noise(m: int, n: int, rank: int = 64, noise: float = 1e-3,
                       seeds=(11, 12, 13), device="cpu", chunk_rows: int = 8192) -> torch.Tensor:
    """A = U V^T + noise * E with U[m x rank], V[n x rank], E[m x n] ~ N(0,1)."""
    U = gaussian_matrix(m, rank, seeds[0], device)
    V = gaussian_matrix(n, rank, seeds[1], device)
    out = gaussian_matrix(m, n, seeds[2], device)
    out.mul_(noise)
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        out[r0:r1].addmm_(U[r0:r1], V.t())
    return out


def rbf_kernel_matrix(n: int, d: int = 64, seed: int = 21, device="cpu",
                      chunk_rows: int = 8192) -> torch.Tensor:
    """K[n x n] = exp(-|x_i - x_j|^2 / (2 sigma^2)) of n points x_i ~ N(0, I_d),
    sigma^2 = |X|_F^2 / n (the paper's choice sigma = |X| / sqrt(n)): a dense
    symmetric positive semi-definite matrix with the structure of the paper's
    RBF kernel matrices, built in place from the Gram matrix."""
    X = gaussian_matrix(n, d, seed, device)
    sq = (X * X).sum(dim=1)
    inv = -0.5 * n / float(sq.sum())
    K = torch.empty((n, n), dtype=torch.float32, device=device)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        blk = K[r0:r1]
        torch.mm(X[r0:r1], X.t(), out=blk)
        blk.mul_(-2.0).add_(sq[r0:r1, None]).add_(sq[None, :]).clamp_(min=0.0)
        blk.mul_(inv).exp_()
    return K


@dataclass(frozen=True)
class Problem:
    m: int
    n: int
    k: int
    dist: int
    seed: int


def batched_problems(count: int = 256, m_lo: int = 1024, m_hi: int = 65536, n_lo: int = 32,
                     n_hi: int = 512, seed: int = 1000) -> list[Problem]:
    """Independent left-sketch problems: m log-uniform in [m_lo, m_hi],
    n uniform in [n_lo, n_hi], k = 2n, dist chosen by a per-problem coin,
    per-problem seeds seed + i."""
    g = _gen("cpu", seed)
    u = torch.rand(count, generator=g, dtype=torch.float64)
    nn = torch.randint(n_lo, n_hi + 1, (count,), generator=g)
    coin = torch.randint(0, 2, (count,), generator=g)
    out = []
    for i in range(count):
        m = int(round(math.exp(math.log(m_lo) + float(u[i]) * (math.log(m_hi) - math.log(m_lo)))))
        n = int(nn[i])
        out.append(Problem(m=m, n=n, k=2 * n, dist=int(coin[i]), seed=seed + i))
    return out


@dataclass(frozen=True)
class Request:
    arrival_s: float   # offset from the start of the stream
    prob: Problem
    row0: int          # first row of the request's A inside the shared source matrix


def serving_requests(count: int = 20000, rate: float = 2000.0, m_lo: int = 1024,
                     m_hi: int = 1 << 18, src_rows: int = 1 << 18, seed: int = 3000
                     ) -> list[Request]:
    """A Poisson stream of left-sketch requests: exponential gaps of mean
    1/rate, shapes drawn as batched_problems (m up to m_hi), and for each a
    random row window of a shared source matrix of src_rows rows."""
    probs = batched_problems(count, m_lo=m_lo, m_hi=m_hi, seed=seed)
    g = _gen("cpu", seed + 1)
    gaps = torch.empty(count, dtype=torch.float64).exponential_(rate, generator=g)
    arrivals = torch.cumsum(gaps, 0) - gaps[0]
    u = torch.rand(count, generator=g, dtype=torch.float64)
    out = []
    for i, p in enumerate(probs):
        row0 = int(float(u[i]) * (src_rows - p.m + 1))
        out.append(Request(arrival_s=float(arrivals[i]), prob=p, row0=min(row0, src_rows - p.m)))
    return out


CONFIGS = {
    "C1": dict(side="left", m=4096, n=256, k=64, dists=(0,), a_seed=A_SEED, s_seed=S_SEED),
    "C2": dict(side="left", m=1 << 20, n=512, k=2048, dists=(1, 0), a_seed=A_SEED,
               s_seed=S_SEED),
    "C3": dict(side="right", m=65536, n=16384, k=256, dists=(0,), a_seed=(11, 12, 13),
               s_seed=S_SEED),
}
