"""Pins of the oracle's tria operator (Section 3.1.2)."""
import numpy as np
import pytest

from oracle.linalg import solve_lower, tria


@pytest.mark.parametrize("n,m", [(1, 1), (3, 5), (4, 4), (8, 16), (10, 14)])
def test_square_root_of_gram(n, m):
    rng = np.random.default_rng(n * 100 + m)
    M = rng.standard_normal((n, m))
    L = tria(M)
    assert L.shape == (n, n)
    np.testing.assert_allclose(L @ L.T, M @ M.T, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.all(np.diag(L) >= 0)
    # a positive definite Gram matrix has a unique Cholesky factor
    np.testing.assert_allclose(L, np.linalg.cholesky(M @ M.T), rtol=1e-10, atol=1e-12)


def test_sum_of_covariances():
    """sqrt(A + B) = tria([sqrt(A), sqrt(B)])."""
    rng = np.random.default_rng(1)
    sA = rng.standard_normal((5, 3))
    sB = np.tril(rng.standard_normal((5, 5)))
    L = tria(np.hstack([sA, sB]))
    np.testing.assert_allclose(L @ L.T, sA @ sA.T + sB @ sB.T, rtol=1e-12)


def test_rank_deficient_and_tall():
    rng = np.random.default_rng(2)
    U = rng.standard_normal((6, 2))
    L = tria(U)                      # tall: padded with zero columns
    np.testing.assert_allclose(L @ L.T, U @ U.T, atol=1e-12)
    assert np.linalg.matrix_rank(L, tol=1e-10) == 2
    Z = tria(np.zeros((3, 4)))
    assert np.all(Z == 0)


def test_solve_lower():
    rng = np.random.default_rng(3)
    Lm = np.tril(rng.standard_normal((5, 5))) + 5 * np.eye(5)
    B = rng.standard_normal((5, 3))
    np.testing.assert_allclose(Lm @ solve_lower(Lm, B), B, atol=1e-12)
