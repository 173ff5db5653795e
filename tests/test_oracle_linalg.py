"""Pins of the oracle's Tria and DownDate (Sec. 2.2) against closed forms,
a different library routine (Cholesky) and the defining properties."""
import numpy as np
import pytest

from oracle.linalg import tria, downdate, NotPositiveDefinite


@pytest.mark.parametrize("n,m", [(1, 1), (2, 5), (5, 10), (5, 15), (7, 7), (10, 10)])
def test_tria_product_lower_and_cholesky(n, m):
    rng = np.random.default_rng(n * 100 + m)
    A = rng.standard_normal((n, m))
    L = tria(A)
    assert L.shape == (n, n)
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.all(np.diag(L) >= 0)
    np.testing.assert_allclose(L @ L.T, A @ A.T, rtol=0, atol=1e-13 * np.abs(A @ A.T).max())
    # full row rank: Tria(A) is the Cholesky factor of A A^T (unique)
    np.testing.assert_allclose(L, np.linalg.cholesky(A @ A.T), atol=1e-11)


def test_tria_2x2_closed_form():
    a, b, c, d = 0.3, -1.2, 2.0, 0.7
    L = tria(np.array([[a, b], [c, d]]))
    l11 = np.hypot(a, b)
    l21 = (a * c + b * d) / l11
    l22 = np.sqrt(c * c + d * d - l21 * l21)
    np.testing.assert_allclose(L, [[l11, 0], [l21, l22]], atol=1e-15)


def test_tria_fewer_columns_than_rows():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((5, 2))
    L = tria(A)
    assert L.shape == (5, 5)
    np.testing.assert_allclose(L @ L.T, A @ A.T, atol=1e-13)


def test_tria_rank_deficient():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((5, 2)) @ rng.standard_normal((2, 10))   # rank 2
    L = tria(A)
    assert np.all(np.isfinite(L))
    np.testing.assert_allclose(L @ L.T, A @ A.T, atol=1e-12)


def test_downdate_scalar_closed_form():
    L = downdate(np.array([[3.0]]), np.array([[2.0]]))
    np.testing.assert_allclose(L, [[np.sqrt(5.0)]], atol=1e-15)


@pytest.mark.parametrize("n,k", [(2, 1), (5, 3), (5, 5)])
def test_downdate_matches_cholesky(n, k):
    rng = np.random.default_rng(10 + n + k)
    B = 0.3 * rng.standard_normal((n, k))
    G = rng.standard_normal((n, n))
    P = B @ B.T + np.eye(n) + 0.1 * G @ G.T
    S = np.linalg.cholesky(P)
    L = downdate(S, B)
    np.testing.assert_allclose(L @ L.T, P - B @ B.T, atol=1e-12)
    np.testing.assert_allclose(L, np.linalg.cholesky(P - B @ B.T), atol=1e-11)


def test_downdate_not_pd_raises():
    S = np.eye(2)
    with pytest.raises(NotPositiveDefinite):
        downdate(S, np.array([[1.5], [0.0]]))
