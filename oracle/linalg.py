"""Tria and DownDate (Sec. 2.2).  Oracle: test infrastructure only.

Readings of the paper taken here:
* Tria(A) is defined through A^T = Q R, Tria(A) = R^T.  The signs of R's rows
  are free; this oracle fixes them so that the diagonal of Tria(A) is >= 0.
  For a rank-deficient A the factor is not unique; any L with L L^T = A A^T is
  correct and only such products are ever compared.
* DownDate(S, B) is the square root of S S^T - B B^T obtained by one rank-1
  Cholesky downdate per column of B (Sec. 2.2, citing Gill-Golub-Murray-
  Saunders).  S must be lower triangular; a non-positive pivot raises.
"""
import numpy as np


class NotPositiveDefinite(ValueError):
    """DownDate met a pivot <= 0: S S^T - B B^T is not positive definite."""


def tria(A):
    """Tria(A) = R^T with A^T = Q R (Sec. 2.2), diagonal made non-negative.

    A is n x m; the result is n x n lower triangular with
    Tria(A) Tria(A)^T = A A^T (property 2 of Sec. 2.2, eq. CCT).
    """
    A = np.asarray(A, dtype=np.float64)
    n, m = A.shape
    R = np.linalg.qr(A.T, mode="r")          # min(m, n) x n, upper trapezoidal
    if R.shape[0] < n:                       # m < n: pad with zero rows of R
        R = np.vstack([R, np.zeros((n - R.shape[0], n))])
    L = R.T.copy()                           # n x n lower triangular
    s = np.sign(np.diag(L))
    s[s == 0] = 1.0
    return L * s[None, :]                    # flip columns: L L^T unchanged


def downdate(S, B):
    """DownDate(S, B): lower L with L L^T = S S^T - B B^T (Sec. 2.2).

    One rank-1 downdate per column b of B: for each pivot k the hyperbolic
    rotation that removes b[k] from L[k, k] is applied to the rest of column k
    and to the rest of b.
    """
    L = np.array(S, dtype=np.float64, copy=True)
    B = np.asarray(B, dtype=np.float64)
    n = L.shape[0]
    if B.ndim == 1:
        B = B[:, None]
    for col in range(B.shape[1]):
        x = B[:, col].copy()
        for k in range(n):
            r2 = L[k, k] ** 2 - x[k] ** 2
            if not (r2 > 0.0) or L[k, k] == 0.0:
                raise NotPositiveDefinite(f"pivot {k}: {r2}")
            r = np.sqrt(r2)
            c = r / L[k, k]
            s = x[k] / L[k, k]
            L[k, k] = r
            L[k + 1:, k] = (L[k + 1:, k] - s * x[k + 1:]) / c
            x[k + 1:] = c * x[k + 1:] - s * L[k + 1:, k]
    return L


def solve_lower(L, B):
    """X with L X = B for lower-triangular L (a library solve used as a step)."""
    import scipy.linalg
    return scipy.linalg.solve_triangular(L, B, lower=True)


def solve_upper(U, B):
    """X with U X = B for upper-triangular U."""
    import scipy.linalg
    return scipy.linalg.solve_triangular(U, B, lower=False)
