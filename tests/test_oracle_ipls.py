"""Pins of the IPLS loop (Alg. 3), pseudo log-likelihood and FD gradient:
exact one-step convergence on linear models; the IEKS fixed point is a
stationary point of the log posterior (Gauss-Newton, Sec. 1); scan orders
agree inside the loop; the FD gradient of a linear model equals the
closed-form derivative of log N(y; mu_y, Sigma_y(theta))."""
import numpy as np
import pytest

from oracle import ipls, models, slr, parallel
from oracle.kalman import sqrt_filter_smoother, sqrt_filter, sqrt_smoother
from paper_2207_00426_gb300 import workloads

THETA = np.log([0.05, 0.01, 0.1])


class LinearCVTheta:
    """Linear CV model with theta = (log sigma, log q)."""
    nx, ny = 4, 2

    def __init__(self, theta, dt=0.1):
        self.theta = np.asarray(theta, dtype=np.float64)
        self.sigma, self.q = np.exp(self.theta)
        base = models.LinearCV(dt=dt, q=self.q, sigma=self.sigma)
        self.F, self.Qm, self.S, self.Hm, self.R, self.SRm = base.matrices()
        self.Q1 = self.Qm / self.q

    def f(self, x): return self.F @ x
    def jac_f(self, x): return self.F
    def SQ(self): return self.S
    def h(self, x): return self.Hm @ x
    def jac_h(self, x): return self.Hm
    def SR(self): return self.SRm
    def branch(self, z, ref): return z


def _lin_data(n, seed=0):
    w = workloads.linear_cv(n=n, seed=seed)
    return w["y"], w["m0"], w["N0"]


@pytest.mark.parametrize("method", ["cubature", "extended"])
def test_ipls_linear_converges_in_one_iteration(method):
    y, m0, N0 = _lin_data(30)
    mdl = LinearCVTheta(np.log([0.5, 0.1]))
    n = y.shape[0]
    tile = lambda A: np.tile(A, (n, 1, 1))
    ref = sqrt_filter_smoother(tile(mdl.F), np.zeros((n, 4)), tile(mdl.S), tile(mdl.Hm),
                               np.zeros((n, 2)), tile(mdl.SRm), y, m0, N0)
    ms1, Ns1, ll1, _ = ipls.ipls(mdl, y, m0, N0, 1, method)
    ms2, Ns2, ll2, _ = ipls.ipls(mdl, y, m0, N0, 2, method)
    np.testing.assert_allclose(ms1, ref[2], atol=1e-10)
    np.testing.assert_allclose(ms2, ms1, atol=1e-10)
    assert abs(ll1 - ref[4]) < 1e-9 and abs(ll2 - ll1) < 1e-9


def test_ieks_fixed_point_is_map():
    d = workloads.ct_sequence(n=40, seed=21)
    ct = models.CTBearings(THETA, dt=d["dt"])
    ms, Ns, _, it = ipls.ipls(ct, d["y"], d["m0"], d["N0"], 200, "extended", tol=1e-13)
    assert it < 200
    Qi = np.linalg.inv(ct.Q())
    Ri = np.linalg.inv(ct.SR() @ ct.SR().T)
    P0i = np.linalg.inv(d["N0"] @ d["N0"].T)
    n = d["y"].shape[0]
    grad = np.zeros_like(ms)
    scale = np.zeros(n + 1)
    grad[0] -= P0i @ (ms[0] - d["m0"])
    for k in range(1, n + 1):
        e = Qi @ (ms[k] - ct.f(ms[k - 1]))
        grad[k] -= e
        grad[k - 1] += ct.jac_f(ms[k - 1]).T @ e
        hk = ct.h(ms[k])
        r = ct.branch(d["y"][k - 1], hk) - hk
        grad[k] += ct.jac_h(ms[k]).T @ Ri @ r
        scale[k] = np.abs(e).max() + np.abs(Ri @ r).max()
    assert np.abs(grad).max() < 1e-7 * scale.max()


def test_scan_order_inside_ipls():
    d = workloads.ct_sequence(n=17, seed=22)
    ct = models.CTBearings(THETA, dt=d["dt"])
    n = 17
    ms = np.tile(d["m0"], (n + 1, 1)); Ns = np.tile(d["N0"], (n + 1, 1, 1))
    for _ in range(3):
        G = slr.linearize(ct, ms, Ns, d["y"], "cubature")
        mf, Nf, _ = sqrt_filter(*G, d["y"], d["m0"], d["N0"])
        mf2, Nf2 = parallel.parallel_sqrt_filter(*G, d["y"], d["m0"], d["N0"])
        np.testing.assert_allclose(mf2, mf, atol=1e-9)
        ms_new, Ns_new = sqrt_smoother(G[0], G[1], G[2], mf, Nf)
        ms2, Ns2 = parallel.parallel_sqrt_smoother(G[0], G[1], G[2], mf, Nf)
        np.testing.assert_allclose(ms2, ms_new, atol=1e-9)
        np.testing.assert_allclose(Ns2 @ np.transpose(Ns2, (0, 2, 1)),
                                   Ns_new @ np.transpose(Ns_new, (0, 2, 1)), atol=1e-10)
        ms, Ns = ms_new, Ns_new


def test_fd_gradient_linear_equals_closed_form():
    n = 25
    y, m0, N0 = _lin_data(n, seed=3)
    theta = np.log([0.6, 0.15])
    g_fd = ipls.nll_grad_fd(LinearCVTheta, theta, y, m0, N0, "extended", h=1e-5, M=2, tol=None)
    mdl = LinearCVTheta(theta)
    # Sigma_y = Tp Tp^T + q Tq Tq^T + sigma^2 I, written from the model directly
    nx, ny = 4, 2
    Tx = [N0]
    Tq = [np.zeros((nx, nx * n))]
    ys = []
    Sy_p = np.zeros((n * ny, n * ny)); Sy_q = np.zeros_like(Sy_p)
    Ap = []; Aq = []
    xp, xq = N0, np.zeros((nx, nx * n))
    Lq1 = np.linalg.cholesky(mdl.Q1)
    for t in range(n):
        xp = mdl.F @ xp
        xq = mdl.F @ xq
        xq[:, nx * t:nx * (t + 1)] += Lq1
        Ap.append(mdl.Hm @ xp); Aq.append(mdl.Hm @ xq)
    Ap = np.vstack(Ap); Aq = np.vstack(Aq)
    S = Ap @ Ap.T + mdl.q * Aq @ Aq.T + mdl.sigma ** 2 * np.eye(n * ny)
    r = y.ravel()                                          # mu_y = 0 (m0 = 0, c = d = 0)
    Si = np.linalg.inv(S)
    a = Si @ r
    dS = [2 * mdl.sigma ** 2 * np.eye(n * ny), mdl.q * Aq @ Aq.T]
    g_ref = np.array([-(-0.5 * np.trace(Si @ D) + 0.5 * a @ D @ a) for D in dS])
    np.testing.assert_allclose(g_fd, g_ref, rtol=1e-7)


def test_fd_gradient_ct_step_consistency():
    d = workloads.ct_sequence(n=20, seed=23)
    kw = dict(dt=d["dt"])
    g1 = ipls.nll_grad_fd(models.CTBearings, THETA, d["y"], d["m0"], d["N0"], "cubature",
                          h=1e-4, tol=1e-13, **kw)
    g2 = ipls.nll_grad_fd(models.CTBearings, THETA, d["y"], d["m0"], d["N0"], "cubature",
                          h=2e-4, tol=1e-13, **kw)
    np.testing.assert_allclose(g1, g2, rtol=1e-5, atol=1e-6 * np.abs(g1).max())


def test_ct_per_sensor_noise_reduces_to_shared():
    """theta = (log s1, log q_c, log q_w, log s2) at s1 = s2 is the model with
    one noise level: same nll, and by the chain rule the shared-sigma
    derivative is the sum of the two per-sensor ones."""
    d = workloads.ct_sequence(n=20, seed=23)
    kw = dict(dt=d["dt"])
    th4 = np.r_[THETA, THETA[0]]
    n3 = ipls.nll(models.CTBearings, THETA, d["y"], d["m0"], d["N0"], "cubature", tol=1e-13, **kw)
    n4 = ipls.nll(models.CTBearings, th4, d["y"], d["m0"], d["N0"], "cubature", tol=1e-13, **kw)
    assert n3 == n4
    g3 = ipls.nll_grad_fd(models.CTBearings, THETA, d["y"], d["m0"], d["N0"], "cubature",
                          h=1e-4, tol=1e-13, **kw)
    g4 = ipls.nll_grad_fd(models.CTBearings, th4, d["y"], d["m0"], d["N0"], "cubature",
                          h=1e-4, tol=1e-13, **kw)
    np.testing.assert_allclose([g4[0] + g4[3], g4[1], g4[2]], g3, rtol=1e-6,
                               atol=1e-7 * np.abs(g3).max())


def test_ct_per_sensor_noise_follows_its_sensor():
    """Relabelling the two sensors, with their noise levels and observation
    columns, leaves the nll unchanged; keeping the noise levels in place
    does not (sqrt(R_11) belongs to the first sensor)."""
    d = workloads.ct_sequence(n=20, seed=29)
    th = np.r_[np.log(0.03), THETA[1:], np.log(0.08)]
    S = models.SENSORS
    kw = dict(dt=d["dt"])
    base = ipls.nll(models.CTBearings, th, d["y"], d["m0"], d["N0"], "cubature", tol=1e-13,
                    sensors=S, **kw)
    swapped = ipls.nll(models.CTBearings, th[[3, 1, 2, 0]], d["y"][:, ::-1], d["m0"], d["N0"],
                       "cubature", tol=1e-13, sensors=S[::-1], **kw)
    wrong = ipls.nll(models.CTBearings, th, d["y"][:, ::-1], d["m0"], d["N0"], "cubature",
                     tol=1e-13, sensors=S[::-1], **kw)
    assert abs(swapped - base) <= 1e-10 * abs(base)
    assert abs(wrong - base) > 1e-3 * abs(base)
