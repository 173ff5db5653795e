"""Pins of the sequential square-root filter / smoother / log-likelihood:
brute-force conditioning of the dense joint Gaussian, the closed-form
steady state of the scalar random walk, and the textbook covariance form."""
import numpy as np
import pytest

from oracle.kalman import (sqrt_filter, sqrt_smoother, sqrt_filter_smoother,
                           cov_filter, cov_smoother)
from paper_2207_00426_gb300.workloads import random_lgssm


def _dense_joint(m):
    """Mean and covariance of (x_0..x_n, y_1..y_n) built by writing every
    variable as an affine function of the independent noises."""
    F, c, SQ, H, d, SR, m0, N0 = (m[k] for k in ("F", "c", "SQ", "H", "d", "SR", "m0", "N0"))
    n, nx, ny = F.shape[0], m0.shape[0], H.shape[1]
    nw = nx * (n + 1) + ny * n                  # x0 noise, q_0..q_{n-1}, v_1..v_n
    Tx = np.zeros((n + 1, nx, nw)); ux = np.zeros((n + 1, nx))
    Tx[0][:, :nx] = N0; ux[0] = m0
    Ty = np.zeros((n, ny, nw)); uy = np.zeros((n, ny))
    for t in range(n):
        Tx[t + 1] = F[t] @ Tx[t]
        Tx[t + 1][:, nx * (t + 1):nx * (t + 2)] += SQ[t]
        ux[t + 1] = F[t] @ ux[t] + c[t]
        Ty[t] = H[t] @ Tx[t + 1]
        off = nx * (n + 1) + ny * t
        Ty[t][:, off:off + ny] += SR[t]
        uy[t] = H[t] @ ux[t + 1] + d[t]
    Tx = Tx.reshape(-1, nw); Ty = Ty.reshape(-1, nw)
    return ux.ravel(), uy.ravel(), Tx, Ty


@pytest.mark.parametrize("nx,ny,n", [(3, 2, 12), (4, 2, 20), (2, 3, 7), (1, 1, 25)])
def test_sqrt_smoother_equals_brute_force(nx, ny, n):
    m = random_lgssm(n, nx, ny, seed=nx * 10 + ny)
    mf, Nf, ms, Ns, ll = sqrt_filter_smoother(m["F"], m["c"], m["SQ"], m["H"], m["d"],
                                              m["SR"], m["y"], m["m0"], m["N0"])
    mux, muy, Tx, Ty = _dense_joint(m)
    Sxy = Tx @ Ty.T
    Syy = Ty @ Ty.T
    Sxx = Tx @ Tx.T
    yv = m["y"].ravel()
    post_m = mux + Sxy @ np.linalg.solve(Syy, yv - muy)
    post_P = Sxx - Sxy @ np.linalg.solve(Syy, Sxy.T)
    np.testing.assert_allclose(ms.ravel(), post_m, atol=1e-9)
    for k in range(n + 1):
        Pk = post_P[k * nx:(k + 1) * nx, k * nx:(k + 1) * nx]
        np.testing.assert_allclose(Ns[k] @ Ns[k].T, Pk, atol=1e-9)
    r = yv - muy
    ll_ref = -0.5 * (len(r) * np.log(2 * np.pi) + np.linalg.slogdet(Syy)[1]
                     + r @ np.linalg.solve(Syy, r))
    assert abs(ll - ll_ref) < 1e-9 * abs(ll_ref)
    # filtering marginal at k conditions on y_1..y_k only
    for k in (1, n // 2, n):
        sel = slice(0, k * ny)
        Sk = Tx[k * nx:(k + 1) * nx] @ Ty[sel].T
        mk = mux[k * nx:(k + 1) * nx] + Sk @ np.linalg.solve(Syy[sel, sel], yv[sel] - muy[sel])
        Pk = (Tx[k * nx:(k + 1) * nx] @ Tx[k * nx:(k + 1) * nx].T
              - Sk @ np.linalg.solve(Syy[sel, sel], Sk.T))
        np.testing.assert_allclose(mf[k], mk, atol=1e-9)
        np.testing.assert_allclose(Nf[k] @ Nf[k].T, Pk, atol=1e-9)


def test_scalar_random_walk_steady_state():
    Q, R, n = 0.3, 2.0, 2000
    rng = np.random.default_rng(5)
    y = rng.standard_normal((n, 1))
    one = np.ones((n, 1, 1))
    mf, Nf, ms, Ns, _ = sqrt_filter_smoother(one, np.zeros((n, 1)), np.sqrt(Q) * one, one,
                                             np.zeros((n, 1)), np.sqrt(R) * one, y,
                                             np.zeros(1), np.eye(1))
    P = (-Q + np.sqrt(Q * Q + 4 * Q * R)) / 2
    Ps = P / (1 + P / (P + Q))
    k = n // 2
    np.testing.assert_allclose(Nf[k, 0, 0] ** 2, P, rtol=1e-12)
    np.testing.assert_allclose(Ns[k, 0, 0] ** 2, Ps, rtol=1e-12)


def test_sqrt_equals_covariance_form():
    m = random_lgssm(40, 5, 2, seed=7)
    Q = m["SQ"] @ np.transpose(m["SQ"], (0, 2, 1))
    R = m["SR"] @ np.transpose(m["SR"], (0, 2, 1))
    mf, Nf, ell = sqrt_filter(m["F"], m["c"], m["SQ"], m["H"], m["d"], m["SR"], m["y"], m["m0"], m["N0"])
    mf2, Pf, _, ell2 = cov_filter(m["F"], m["c"], Q, m["H"], m["d"], R, m["y"], m["m0"], m["N0"] @ m["N0"].T)
    np.testing.assert_allclose(mf, mf2, atol=1e-10)
    np.testing.assert_allclose(Nf @ np.transpose(Nf, (0, 2, 1)), Pf, atol=1e-10)
    np.testing.assert_allclose(ell, ell2, atol=1e-10)
    ms, Ns = sqrt_smoother(m["F"], m["c"], m["SQ"], mf, Nf)
    ms2, Ps = cov_smoother(m["F"], m["c"], Q, mf2, Pf)
    np.testing.assert_allclose(ms, ms2, atol=1e-10)
    np.testing.assert_allclose(Ns @ np.transpose(Ns, (0, 2, 1)), Ps, atol=1e-10)
