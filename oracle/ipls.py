"""Iterated posterior linearisation (Alg. 3), pseudo log-likelihood
(Sec. 5.1) and its gradient (Sec. 5.2).  Oracle: test infrastructure only.

Readings:
* the initial nominal trajectory (Alg. 3 input, not specified) is the prior
  broadcast to every step: m^{s,(0)}_k = m_0, N^{s,(0)}_k = N_0;
* the pseudo log-likelihood is the sum of the l_k of the filter run in the
  last iteration, i.e. on Gamma^(M) linearised at the nominal trajectory of
  iteration M-1 (at a fixed point the two agree);
* the gradient is the total derivative through the fixed point (eq.
  implicity_function_theorem); the oracle obtains it by central finite
  differences of the converged pseudo log-likelihood.
"""
import numpy as np

from .kalman import cov_filter, cov_smoother, sqrt_filter, sqrt_smoother
from .slr import linearize, linearize_std


def ipls(model, y, m0, N0, M, method="cubature", init=None, tol=None):
    """Alg. 3: M times {linearise all steps (Sec. 4.2/4.3); square-root
    filter (Alg. 1); square-root smoother (Alg. 2)}.  With tol set, stops
    early once max_k |m^{s,(i)}_k - m^{s,(i-1)}_k|_inf < tol.
    Returns ms, Ns, loglik, iterations."""
    n = y.shape[0]
    if init is None:
        ms = np.tile(m0, (n + 1, 1))
        Ns = np.tile(N0, (n + 1, 1, 1))
    else:
        ms, Ns = (np.array(a, dtype=np.float64) for a in init)
    loglik = np.nan
    it = 0
    for it in range(1, M + 1):
        G = linearize(model, ms, Ns, y, method)
        mf, Nf, ell = sqrt_filter(*G, y, m0, N0)
        ms_new, Ns_new = sqrt_smoother(G[0], G[1], G[2], mf, Nf)
        loglik = float(np.sum(ell))
        delta = np.max(np.abs(ms_new - ms))
        ms, Ns = ms_new, Ns_new
        if tol is not None and delta < tol:
            break
    return ms, Ns, loglik, it


def nll(model_cls, theta, y, m0, N0, method="cubature", M=200, tol=1e-12,
        init=None, **model_kw):
    """Negative pseudo log-likelihood at the fixed point of Alg. 3."""
    model = model_cls(theta, **model_kw)
    _, _, ll, _ = ipls(model, y, m0, N0, M, method, init=init, tol=tol)
    return -ll


def nll_grad_fd(model_cls, theta, y, m0, N0, method="cubature", h=1e-4,
                M=200, tol=1e-12, init=None, **model_kw):
    """Central finite differences of nll in each component of theta."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros_like(theta)
    for j in range(theta.size):
        e = np.zeros_like(theta)
        e[j] = h
        fp = nll(model_cls, theta + e, y, m0, N0, method, M, tol, init, **model_kw)
        fm = nll(model_cls, theta - e, y, m0, N0, method, M, tol, init, **model_kw)
        g[j] = (fp - fm) / (2.0 * h)
    return g


def ipls_std(model, y, m0, P0, M, init=None, tol=None):
    """Alg. 3 in the standard (covariance) form: M times {covariance-form
    cubature linearisation; covariance Kalman filter; covariance RTS
    smoother}.  Same readings and stopping rule as ipls.  Returns ms, Ps,
    loglik, iterations."""
    n = y.shape[0]
    if init is None:
        ms = np.tile(m0, (n + 1, 1))
        Ps = np.tile(P0, (n + 1, 1, 1))
    else:
        ms, Ps = (np.array(a, dtype=np.float64) for a in init)
    loglik = np.nan
    it = 0
    for it in range(1, M + 1):
        F, c, Q, H, d, R = linearize_std(model, ms, Ps, y)
        mf, Pf, _, ell = cov_filter(F, c, Q, H, d, R, y, m0, P0)
        ms_new, Ps_new = cov_smoother(F, c, Q, mf, Pf)
        loglik = float(np.sum(ell))
        delta = np.max(np.abs(ms_new - ms))
        ms, Ps = ms_new, Ps_new
        if tol is not None and delta < tol:
            break
    return ms, Ps, loglik, it

