"""Sequential Kalman filter and RTS smoother, square-root and covariance forms.

Oracle: test infrastructure only.

The parallel filter of Alg. 1 produces, as its prefixes, exactly the
sequential filtering distributions (Sec. 2.1: a_1 x ... x a_k recovers
p(x_k | y_{1:k})), and the reverse scan of Alg. 2 the smoothing
distributions.  So for a given linear(ised) model the oracle of both scans is
the plain sequential recursion written here.

Array conventions (time index t = 0 .. n-1, model of eq. linear-model):
  F[t], c[t], SQ[t]  transition x_{t+1} = F[t] x_t + c[t] + q,
                     q ~ N(0, SQ[t] SQ[t]^T)          (F_{k-1}, c_{k-1}, S_Lambda_{k-1})
  H[t], d[t], SR[t]  observation y_{t+1} = H[t] x_{t+1} + d[t] + v,
                     v ~ N(0, SR[t] SR[t]^T)          (H_k, d_k, S_Omega_k)
  y[t]               y_{t+1}
Outputs are indexed k = 0 .. n (k = 0 is the prior).
"""
import numpy as np

from .linalg import tria, solve_lower, solve_upper

LOG2PI = np.log(2.0 * np.pi)


def sqrt_filter(F, c, SQ, H, d, SR, y, m0, N0):
    """Sequential square-root Kalman filter.

    Each step is the k = 1 construction of Lemma 1 / Table 1 (right column)
    with (m_0, N_0) replaced by the previous filtering result:
      m^- = F m + c,  N^- = Tria([F N, S_Lambda]),
      Psi = Tria([[H N^-, S_Omega], [N^-, 0]])  (eq. sqrt-filter-step1),
      Y = Psi_11, K = Psi_21 Psi_11^{-1}, m = m^- + K (y - H m^- - d),
      N = Psi_22.
    The log-likelihood term (Sec. 5.1) is
      l_k = log N(y_k; H m^- + d, Y Y^T).
    Returns mf (n+1, nx), Nf (n+1, nx, nx), ell (n,).
    """
    n = y.shape[0]
    nx = m0.shape[0]
    ny = y.shape[1]
    mf = np.zeros((n + 1, nx))
    Nf = np.zeros((n + 1, nx, nx))
    ell = np.zeros(n)
    mf[0] = m0
    Nf[0] = N0
    for t in range(n):
        m_pred = F[t] @ mf[t] + c[t]
        N_pred = tria(np.hstack([F[t] @ Nf[t], SQ[t]]))
        top = np.hstack([H[t] @ N_pred, SR[t]])
        bot = np.hstack([N_pred, np.zeros((nx, ny))])
        Psi = tria(np.vstack([top, bot]))
        Y = Psi[:ny, :ny]
        Psi21 = Psi[ny:, :ny]
        Psi22 = Psi[ny:, ny:]
        K = solve_upper(Y.T, Psi21.T).T                 # K Y = Psi21
        v = y[t] - H[t] @ m_pred - d[t]
        mf[t + 1] = m_pred + K @ v
        Nf[t + 1] = Psi22
        e = solve_lower(Y, v)
        ell[t] = -0.5 * (ny * LOG2PI + 2.0 * np.sum(np.log(np.abs(np.diag(Y))))
                         + e @ e)
    return mf, Nf, ell


def sqrt_smoother(F, c, SQ, mf, Nf):
    """Sequential square-root RTS smoother.

    For k = n-1 .. 0 the Lemma 3 quantities (eq. smooth-init-2, Table 4 right)
      Phi = Tria([[F_k N^f_k, S_Lambda_k], [N^f_k, 0]]),
      E_k = Phi_21 Phi_11^{-1},  g_k = m^f_k - E_k (F_k m^f_k + c_k),
      D_k = Phi_22
    are combined with the smoothing result at k+1 by Lemma 4 / Table 5 with
    E_{k+1:n} = 0:  m^s_k = E_k m^s_{k+1} + g_k,
                    N^s_k = Tria([E_k N^s_{k+1}, D_k]).
    Returns ms (n+1, nx), Ns (n+1, nx, nx).
    """
    n = F.shape[0]
    nx = mf.shape[1]
    ms = np.zeros_like(mf)
    Ns = np.zeros_like(Nf)
    ms[n] = mf[n]
    Ns[n] = Nf[n]
    for k in range(n - 1, -1, -1):
        top = np.hstack([F[k] @ Nf[k], SQ[k]])
        bot = np.hstack([Nf[k], np.zeros((nx, nx))])
        Phi = tria(np.vstack([top, bot]))
        Phi11 = Phi[:nx, :nx]
        Phi21 = Phi[nx:, :nx]
        Phi22 = Phi[nx:, nx:]
        E = solve_upper(Phi11.T, Phi21.T).T             # E Phi11 = Phi21
        g = mf[k] - E @ (F[k] @ mf[k] + c[k])
        ms[k] = E @ ms[k + 1] + g
        Ns[k] = tria(np.hstack([E @ Ns[k + 1], Phi22]))
    return ms, Ns


def cov_filter(F, c, Q, H, d, R, y, m0, P0):
    """Textbook covariance Kalman filter (Table 1 left column, one step at a
    time): predict m^- = F m + c, P^- = F P F^T + Lambda; update with
    S = H P^- H^T + Omega, K = P^- H^T S^{-1}.  Q and R are covariances."""
    n = y.shape[0]
    nx = m0.shape[0]
    mf = np.zeros((n + 1, nx))
    Pf = np.zeros((n + 1, nx, nx))
    Pp = np.zeros((n, nx, nx))
    ell = np.zeros(n)
    mf[0] = m0
    Pf[0] = P0
    for t in range(n):
        m_pred = F[t] @ mf[t] + c[t]
        P_pred = F[t] @ Pf[t] @ F[t].T + Q[t]
        S = H[t] @ P_pred @ H[t].T + R[t]
        K = np.linalg.solve(S, H[t] @ P_pred).T
        v = y[t] - H[t] @ m_pred - d[t]
        mf[t + 1] = m_pred + K @ v
        Pf[t + 1] = P_pred - K @ S @ K.T
        Pp[t] = P_pred
        ell[t] = -0.5 * (len(v) * LOG2PI + np.linalg.slogdet(S)[1]
                         + v @ np.linalg.solve(S, v))
    return mf, Pf, Pp, ell


def cov_smoother(F, c, Q, mf, Pf):
    """Textbook covariance RTS smoother (Table 4 left column composed with
    Table 5 left column): G = P^f F^T (F P^f F^T + Lambda)^{-1},
    m^s_k = m^f_k + G (m^s_{k+1} - F m^f_k - c),
    P^s_k = P^f_k + G (P^s_{k+1} - P^-_{k+1}) G^T."""
    n = F.shape[0]
    ms = np.zeros_like(mf)
    Ps = np.zeros_like(Pf)
    ms[n] = mf[n]
    Ps[n] = Pf[n]
    for k in range(n - 1, -1, -1):
        P_pred = F[k] @ Pf[k] @ F[k].T + Q[k]
        G = np.linalg.solve(P_pred, F[k] @ Pf[k]).T
        ms[k] = mf[k] + G @ (ms[k + 1] - F[k] @ mf[k] - c[k])
        Ps[k] = Pf[k] + G @ (Ps[k + 1] - P_pred) @ G.T
    return ms, Ps


def sqrt_filter_smoother(F, c, SQ, H, d, SR, y, m0, N0):
    """Sequential square-root filter then smoother on one linear(ised) model.
    Returns (mf, Nf, ms, Ns, loglik) with loglik = sum_k l_k (Sec. 5.1)."""
    mf, Nf, ell = sqrt_filter(F, c, SQ, H, d, SR, y, m0, N0)
    ms, Ns = sqrt_smoother(F, c, SQ, mf, Nf)
    return mf, Nf, ms, Ns, float(np.sum(ell))
