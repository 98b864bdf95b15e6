"""Pins of the oracle's Nystrom pair (B = A Omega, C = Omega^T B, Sec. 5)
against other routes to the same numbers: associativity through the left
sketch (C = (S A) S^T), symmetry of C for symmetric A, the brute-force
triple product on tiny inputs, and exact recovery of a PSD matrix of rank
below k by the Nystrom formula."""
import numpy as np
import pytest

import oracle


def _sym(n, seed):
    g = np.random.default_rng(seed).standard_normal((n, n))
    return ((g + g.T) / 2).astype(np.float32)


@pytest.mark.parametrize("dist,prec", [(0, 0), (1, 0), (0, 1), (2, 0)])
def test_associativity_and_symmetry(dist, prec):
    n, k = 40, 7
    A = _sym(n, 1)
    B, C = oracle.nystrom(3, dist, prec, k, A)
    # other order: (S A) S^T through the left then the right sketch
    SA = oracle.apply_left(3, dist, prec, k, A)            # k x n, FP64
    S = oracle.materialize_scaled(3, dist, prec, k, 0, 0, k, n)
    assert np.allclose(SA @ S.T, C, rtol=1e-12, atol=1e-12)
    assert np.allclose(C, C.T, rtol=1e-12, atol=1e-12)
    assert np.allclose(B, A.astype(np.float64) @ S.T, rtol=1e-12, atol=1e-12)


def test_brute_force_tiny():
    n, k = 5, 3
    A = _sym(n, 2)
    B, C = oracle.nystrom(9, 0, 0, k, A)
    g = oracle.generate(9, 0, 0, 0, 0, k, n).astype(np.float64)
    s = float(oracle.scale(k))
    want = np.zeros((k, k))
    for i in range(k):
        for j in range(k):
            want[i, j] = sum(s * g[i, a] * A[a, b] * s * g[j, b] for a in range(n) for b in range(n))
    assert np.allclose(C, want, rtol=1e-12, atol=1e-13)


def test_low_rank_psd_recovered():
    # A = U U^T of rank 4 < k: A = B C^+ B^T exactly (up to FP64 rounding)
    n, k, rank = 60, 10, 4
    U = np.random.default_rng(5).standard_normal((n, rank)).astype(np.float32)
    A = (U.astype(np.float64) @ U.T.astype(np.float64)).astype(np.float32)
    B, C = oracle.nystrom(11, 0, 0, k, A)
    rec = B @ np.linalg.pinv(C, rcond=1e-10) @ B.T
    assert np.linalg.norm(rec - A) / np.linalg.norm(A) < 1e-6
