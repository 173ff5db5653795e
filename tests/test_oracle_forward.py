"""Pins of the oracle's forward-mode gradient (oracle/forward.py), the second
route to d nll / d theta next to the central differences of
ipls.nll_grad_fd:

- the Tria tangent against central differences of Tria on random
  full-row-rank blocks (its definition through the Cholesky factor);
- the CT model's noise-factor derivatives against differences of SQ, SR;
- a linear model: the forward-mode gradient equals the closed-form
  derivative of log N(y; mu_y, Sigma_y(theta)) of the dense joint Gaussian;
- the CT model (three and four parameters): forward mode and central
  differences of the converged pseudo log-likelihood agree to ~1e-6."""
import numpy as np
import pytest

from oracle import forward, ipls, models
from oracle.linalg import tria
from paper_2207_00426_gb300 import workloads

THETA = np.log([0.05, 0.01, 0.1])


@pytest.mark.parametrize("shape", [(5, 10), (7, 12), (2, 7)])
def test_tria_tangent_matches_differences(shape):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape)
    dA = rng.standard_normal(shape + (2,))
    L, dL = forward.tria_jvp(A, dA)
    h = 1e-6
    for p in range(2):
        fd = (tria(A + h * dA[:, :, p]) - tria(A - h * dA[:, :, p])) / (2 * h)
        np.testing.assert_allclose(dL[:, :, p], fd, rtol=0, atol=1e-7 * np.abs(fd).max())
    np.testing.assert_allclose(L, tria(A))


@pytest.mark.parametrize("theta", [THETA, np.r_[np.log(0.03), THETA[1:], np.log(0.08)]])
def test_ct_noise_factor_derivatives(theta):
    m = models.CTBearings(theta, dt=0.01)
    dSQ, dSR = m.dSQ_dtheta(), m.dSR_dtheta()
    h = 1e-6
    for j in range(theta.size):
        e = np.zeros_like(theta)
        e[j] = h
        mp, mm = models.CTBearings(theta + e, dt=0.01), models.CTBearings(theta - e, dt=0.01)
        np.testing.assert_allclose(dSQ[:, :, j], (mp.SQ() - mm.SQ()) / (2 * h), atol=1e-9)
        np.testing.assert_allclose(dSR[:, :, j], (mp.SR() - mm.SR()) / (2 * h), atol=1e-9)


class LinearCVTheta:
    """Linear constant-velocity model with theta = (log sigma, log q) and the
    parameter derivatives of its noise factors."""
    nx, ny = 4, 2

    def __init__(self, theta, dt=0.1):
        self.theta = np.asarray(theta, dtype=np.float64)
        self.sigma, self.q = np.exp(self.theta)
        base = models.LinearCV(dt=dt, q=self.q, sigma=self.sigma)
        self.F, self.Qm, self.S, self.Hm, self.R, self.SRm = base.matrices()

    def f(self, x): return self.F @ x
    def jac_f(self, x): return self.F
    def SQ(self): return self.S
    def h(self, x): return self.Hm @ x
    def jac_h(self, x): return self.Hm
    def SR(self): return self.SRm
    def branch(self, z, ref): return z

    def dSQ_dtheta(self):
        D = np.zeros((4, 4, 2))
        D[:, :, 1] = 0.5 * self.S
        return D

    def dSR_dtheta(self):
        D = np.zeros((2, 2, 2))
        D[:, :, 0] = self.SRm
        return D


def _closed_form_grad(mdl, y, N0):
    """d(-log N(y; 0, Sigma_y))/d theta for the linear model with m0 = 0,
    built from the dense joint Gaussian: Sigma_y = Ap Ap^T + q Aq Aq^T +
    sigma^2 I (prior part, process-noise part, observation noise)."""
    n = y.shape[0]
    nx, ny = 4, 2
    xp, xq = N0, np.zeros((nx, nx * n))
    Lq1 = np.linalg.cholesky(mdl.Qm / mdl.q)
    Ap, Aq = [], []
    for t in range(n):
        xp = mdl.F @ xp
        xq = mdl.F @ xq
        xq[:, nx * t:nx * (t + 1)] += Lq1
        Ap.append(mdl.Hm @ xp)
        Aq.append(mdl.Hm @ xq)
    Ap, Aq = np.vstack(Ap), np.vstack(Aq)
    S = Ap @ Ap.T + mdl.q * Aq @ Aq.T + mdl.sigma ** 2 * np.eye(n * ny)
    Si = np.linalg.inv(S)
    a = Si @ y.ravel()
    dS = [2 * mdl.sigma ** 2 * np.eye(n * ny), mdl.q * Aq @ Aq.T]
    nll = 0.5 * (n * ny * np.log(2 * np.pi) + np.linalg.slogdet(S)[1] + y.ravel() @ a)
    return nll, np.array([-(-0.5 * np.trace(Si @ D) + 0.5 * a @ D @ a) for D in dS])


def test_forward_gradient_linear_equals_closed_form():
    w = workloads.linear_cv(n=25, seed=3)
    mdl = LinearCVTheta(np.log([0.6, 0.15]))
    nll, g, it = forward.nll_grad_forward(mdl, w["y"], w["m0"], w["N0"])
    nll_ref, g_ref = _closed_form_grad(mdl, w["y"], w["N0"])
    assert it <= 3                        # linear: the fixed point after one iteration
    np.testing.assert_allclose(g, g_ref, rtol=1e-9)
    assert abs(nll - nll_ref) < 1e-9 * abs(nll_ref)


@pytest.mark.parametrize("theta", [THETA, np.r_[np.log(0.03), THETA[1:], np.log(0.08)]])
def test_forward_gradient_ct_matches_central_differences(theta):
    d = workloads.ct_sequence(n=20, seed=23)
    mdl = models.CTBearings(theta, dt=d["dt"])
    nll, g, it = forward.nll_grad_forward(mdl, d["y"], d["m0"], d["N0"], tol=1e-12)
    g_fd = ipls.nll_grad_fd(models.CTBearings, theta, d["y"], d["m0"], d["N0"], "cubature",
                            h=1e-4, tol=1e-13, dt=d["dt"])
    assert it < 200
    np.testing.assert_allclose(g, g_fd, rtol=1e-6, atol=1e-6 * np.abs(g_fd).max())
    nll_fp = ipls.nll(models.CTBearings, theta, d["y"], d["m0"], d["N0"], "cubature", tol=1e-13,
                      dt=d["dt"])
    assert abs(nll - nll_fp) < 1e-9 * abs(nll_fp)
