"""Pins for the oracle's sketch products (the definition B = A Omega of
Sec. 1 / Sec. 3, and its transposed left form S A): brute force against
numpy's matmul on the materialized matrix, special inputs (identity, unit
vectors), the transposition identity, and the moment invariants of a
scaled Gaussian / Rademacher sketch over many seeds."""
import numpy as np
import pytest

G, R = 0, 1


def rand_a(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape).astype(np.float32)


@pytest.mark.parametrize("dist", [G, R])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("k,m,n", [(1, 1, 1), (3, 5, 2), (8, 8, 8), (4, 7, 3), (5, 130, 6)])
def test_left_brute_force(orc, dist, prec, k, m, n):
    A = rand_a((m, n), k * 100 + m * 10 + n)
    S = orc.materialize_scaled(17, dist, prec, k, 0, 0, k, m)
    Y = orc.apply_left(17, dist, prec, k, A, nthreads=2)
    np.testing.assert_allclose(Y, S @ A.astype(np.float64), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("dist", [G, R])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("k,m,n", [(1, 1, 1), (2, 3, 5), (8, 8, 8), (3, 4, 131)])
def test_right_brute_force(orc, dist, prec, k, m, n):
    A = rand_a((m, n), 7 + k + m + n)
    S = orc.materialize_scaled(23, dist, prec, k, 0, 0, k, n)
    Y = orc.apply_right(23, dist, prec, k, A, nthreads=3)
    np.testing.assert_allclose(Y, A.astype(np.float64) @ S.T, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("dist", [G, R])
def test_transposition_identity(orc, dist):
    A = rand_a((37, 300), 1)
    right = orc.apply_right(9, dist, 0, 12, A)
    left = orc.apply_left(9, dist, 0, 12, np.ascontiguousarray(A.T))
    np.testing.assert_array_equal(right, left.T)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_identity_input_gives_scaled_matrix(orc, prec):
    m, k = 64, 16
    Y = orc.apply_left(31, G, prec, k, np.eye(m, dtype=np.float32))
    np.testing.assert_array_equal(Y, orc.materialize_scaled(31, G, prec, k, 0, 0, k, m))


def test_unit_vector_picks_a_column(orc):
    m, k, j = 50, 10, 37
    e = np.zeros((m, 1), np.float32)
    e[j, 0] = 1
    Y = orc.apply_left(4, R, 0, k, e)
    np.testing.assert_array_equal(Y[:, 0], orc.materialize_scaled(4, R, 0, k, 0, j, k, 1)[:, 0])


def test_column_and_row_subsets(orc):
    A = rand_a((40, 33), 2)
    full = orc.apply_left(5, G, 0, 9, A)
    cols = np.array([0, 32, 7, 7, 15])
    np.testing.assert_array_equal(orc.apply_left(5, G, 0, 9, A, cols=cols), full[:, cols])
    fr = orc.apply_right(5, G, 0, 9, A)
    rows = np.array([39, 0, 21])
    np.testing.assert_array_equal(orc.apply_right(5, G, 0, 9, A, rows=rows), fr[rows])


def test_threads_do_not_change_results(orc):
    A = rand_a((300, 17), 3)
    a = orc.apply_left(6, G, 0, 33, A, nthreads=1)
    b = orc.apply_left(6, G, 0, 33, A, nthreads=7)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dist", [G, R])
def test_norm_preserved_in_expectation(orc, dist):
    # E ||S x||^2 = ||x||^2 for S with i.i.d. entries of variance 1/k
    m, k, trials = 48, 8, 3000
    x = rand_a((m, 1), 8)
    vals = np.array([np.sum(orc.apply_left(1000 + t, dist, 0, k, x, nthreads=1) ** 2)
                     for t in range(trials)])
    nx2 = float(np.sum(x.astype(np.float64) ** 2))
    se = vals.std(ddof=1) / np.sqrt(trials)
    assert abs(vals.mean() - nx2) < 5 * se


@pytest.mark.parametrize("dist", [G, R])
def test_expected_gram_is_identity(orc, dist):
    # E[S^T S] = I for the scaled matrix
    k, m, trials = 8, 12, 2000
    acc = np.zeros((m, m))
    acc2 = np.zeros((m, m))
    for t in range(trials):
        S = orc.materialize_scaled(5000 + t, dist, 0, k, 0, 0, k, m)
        gram = S.T @ S
        acc += gram
        acc2 += gram**2
    mean = acc / trials
    se = np.sqrt(np.maximum(acc2 / trials - mean**2, 1e-30) / trials)
    assert np.all(np.abs(mean - np.eye(m)) < 6 * se + 1e-12)
    if dist == R:
        S = orc.materialize_scaled(1, R, 0, 16, 0, 0, 16, m)
        np.testing.assert_array_equal(np.diag(S.T @ S), np.ones(m))


def test_bad_arguments_raise(orc):
    with pytest.raises(ValueError):
        orc.apply_left(1, G, 0, 0, rand_a((4, 4), 0))


def test_row_blocks_match_full(orc):
    A = rand_a((70, 9), 12)
    full = orc.apply_left(2, G, 0, 20, A)
    np.testing.assert_array_equal(orc.apply_left(2, G, 0, 20, A, rows=(5, 11)), full[5:16])
    np.testing.assert_array_equal(orc.apply_left(2, G, 0, 20, A, rows=(19, 1), cols=[3, 1]),
                                  full[19:20, [3, 1]])
    with pytest.raises(ValueError):
        orc.apply_left(2, G, 0, 20, A, rows=(15, 6))
