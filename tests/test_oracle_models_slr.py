"""Pins of the CT model (Jacobians vs central differences, series vs
high-precision closed forms, noise factor vs Cholesky) and of the SLR
(exact on linear functions; cubature exact for quadratics; DownDate form
equal to the residual form; bearing branches)."""
import mpmath
import numpy as np
import pytest

from oracle import models, slr
from oracle.linalg import tria

THETA = np.log([0.05, 0.01, 0.1])


def _fd_jac(fun, x, h=1e-6):
    J = np.zeros((len(fun(x)), len(x)))
    for i in range(len(x)):
        e = np.zeros_like(x); e[i] = h
        J[:, i] = (fun(x + e) - fun(x - e)) / (2 * h)
    return J


@pytest.mark.parametrize("w", [0.0, 0.05, -0.09, 0.5, 5.0, 12.0, -20.0])
@pytest.mark.parametrize("dt", [0.01, 0.3])
def test_ct_jacobian_matches_central_differences(w, dt):
    m = models.CTBearings(THETA, dt=dt)
    x = np.array([0.3, -1.2, 1.1, -0.4, w])
    np.testing.assert_allclose(m.jac_f(x), _fd_jac(m.f, x), atol=1e-8)
    np.testing.assert_allclose(m.jac_h(x), _fd_jac(m.h, x), atol=1e-8)


@pytest.mark.parametrize("a", [1e-5, 9.99e-4, 1.001e-3, 0.02, 0.0999, 0.1001, 0.7])
def test_turn_coefficients_match_high_precision(a):
    mpmath.mp.dps = 40
    dt = 0.01
    w = a / dt
    S, C = models._turn_coeffs(w, dt)
    dS, dC = models._turn_coeff_derivs(w, dt)
    A = mpmath.mpf(a)
    S_ref = dt * mpmath.sin(A) / A
    C_ref = dt * (1 - mpmath.cos(A)) / A
    dS_ref = dt * dt * (A * mpmath.cos(A) - mpmath.sin(A)) / A ** 2
    dC_ref = dt * dt * (A * mpmath.sin(A) - (1 - mpmath.cos(A))) / A ** 2
    assert abs(S - float(S_ref)) <= 1e-15 * abs(float(S_ref))
    assert abs(C - float(C_ref)) <= 1e-13 * abs(float(C_ref))
    assert abs(dS - float(dS_ref)) <= 1e-12 * abs(float(dS_ref))
    assert abs(dC - float(dC_ref)) <= 1e-12 * abs(float(dC_ref))


def test_ct_constant_velocity_limit_and_speed():
    m = models.CTBearings(THETA, dt=0.01)
    x = np.array([1.0, 2.0, 0.5, -0.7, 0.0])
    np.testing.assert_allclose(m.f(x)[:2], x[:2] + 0.01 * x[2:4], atol=1e-16)
    x[4] = 3.0
    fx = m.f(x)
    assert abs(np.hypot(*fx[2:4]) - np.hypot(*x[2:4])) < 1e-15


def test_ct_noise_factor_is_cholesky_of_Q():
    m = models.CTBearings(THETA, dt=0.01)
    np.testing.assert_allclose(m.SQ() @ m.SQ().T, m.Q(), rtol=1e-13, atol=1e-20)
    np.testing.assert_allclose(m.SQ(), np.linalg.cholesky(m.Q()), rtol=1e-9, atol=1e-15)


class _Linear:
    nx, ny = 3, 2

    def __init__(self, seed=0):
        rng = np.random.default_rng(seed)
        self.A = rng.standard_normal((3, 3))
        self.u = rng.standard_normal(3)
        self.Hm = rng.standard_normal((2, 3))
        self.dv = rng.standard_normal(2)
        self.S = np.tril(rng.standard_normal((3, 3))) + 2 * np.eye(3)
        self.R = np.tril(rng.standard_normal((2, 2))) + 2 * np.eye(2)

    def f(self, x): return self.A @ x + self.u
    def jac_f(self, x): return self.A
    def SQ(self): return self.S
    def h(self, x): return self.Hm @ x + self.dv
    def jac_h(self, x): return self.Hm
    def SR(self): return self.R
    def branch(self, z, ref): return z


def test_slr_exact_on_linear_functions():
    lm = _Linear()
    rng = np.random.default_rng(1)
    m = rng.standard_normal(3)
    N = np.tril(rng.standard_normal((3, 3))) + 1.5 * np.eye(3)
    for F, c, S in (slr.transition_cubature(lm, m, N), slr.transition_taylor(lm, m)):
        np.testing.assert_allclose(F, lm.A, atol=1e-12)
        np.testing.assert_allclose(c, lm.u, atol=1e-12)
        np.testing.assert_allclose(S @ S.T, lm.S @ lm.S.T, atol=1e-12)
    y = rng.standard_normal(2)
    for H, d, S in (slr.observation_cubature(lm, m, N, y), slr.observation_taylor(lm, m, y)):
        np.testing.assert_allclose(H, lm.Hm, atol=1e-12)
        np.testing.assert_allclose(d, lm.dv, atol=1e-12)
        np.testing.assert_allclose(S @ S.T, lm.R @ lm.R.T, atol=1e-12)


class _Quadratic(_Linear):
    def __init__(self):
        super().__init__(3)
        rng = np.random.default_rng(4)
        B = rng.standard_normal((3, 3, 3))
        self.B = B + np.transpose(B, (0, 2, 1))

    def f(self, x): return np.einsum("ijk,j,k->i", self.B, x, x)


def test_cubature_exact_for_quadratics():
    """E[x^T B x] = tr(B P) + m^T B m and Cov(x^T B x, x) = 2 P B m for
    Gaussian x; the degree-3 rule reproduces both."""
    q = _Quadratic()
    rng = np.random.default_rng(2)
    m = rng.standard_normal(3)
    N = np.tril(rng.standard_normal((3, 3))) + 1.5 * np.eye(3)
    Pm = N @ N.T
    F, c, _ = slr.transition_cubature(q, m, N)
    mean = np.array([np.trace(q.B[i] @ Pm) + m @ q.B[i] @ m for i in range(3)])
    Fref = np.array([2 * q.B[i] @ m for i in range(3)])      # Cov(f_i, x) P^{-1}
    np.testing.assert_allclose(F, Fref, atol=1e-11)
    np.testing.assert_allclose(c + F @ m, mean, atol=1e-11)


def test_downdate_form_equals_residual_form():
    ct = models.CTBearings(THETA, dt=0.01)
    m = np.array([0.4, -0.8, 1.0, 0.5, 2.0])
    N = np.diag([0.1, 0.12, 0.2, 0.15, 0.5])
    N[3, 1] = 0.03; N[4, 2] = -0.1
    X, w = slr.cubature_points(m, N)
    Zs = np.array([ct.f(x) for x in X])
    F, c, S = slr.transition_cubature(ct, m, N)
    S2 = slr.residual_noise_factor(m, N, Zs, w, ct.SQ(), F)
    np.testing.assert_allclose(S @ S.T, S2 @ S2.T, rtol=1e-9, atol=1e-15)
    Xs = np.array([ct.branch(ct.h(x), ct.h(m)) for x in X])
    H, d, So = slr.observation_cubature(ct, m, N, ct.h(m))
    So2 = slr.residual_noise_factor(m, N, Xs, w, ct.SR(), H)
    np.testing.assert_allclose(So @ So.T, So2 @ So2.T, rtol=1e-9, atol=1e-15)


def test_cubature_tends_to_taylor_for_small_covariance():
    ct = models.CTBearings(THETA, dt=0.01)
    m = np.array([0.4, -0.8, 1.0, 0.5, 2.0])
    N = 1e-5 * np.eye(5)
    F, c, _ = slr.transition_cubature(ct, m, N)
    np.testing.assert_allclose(F, ct.jac_f(m), atol=1e-8)
    H, d, _ = slr.observation_cubature(ct, m, N, ct.h(m))
    np.testing.assert_allclose(H, ct.jac_h(m), atol=1e-6)


def test_bearing_branch_across_the_cut():
    """Target left of sensor 1 at its height: bearings straddle +-pi."""
    ct = models.CTBearings(THETA, dt=0.01)
    m = np.array([-3.0, 0.5 + 1e-3, 0.0, 0.0, 0.0])
    N = 0.05 * np.eye(5)
    y = np.array([-np.pi + 0.01, ct.h(m)[1]])          # measured across the cut
    for H, d, _ in (slr.observation_cubature(ct, m, N, y), slr.observation_taylor(ct, m, y)):
        r = y - H @ m - d
        np.testing.assert_allclose(r, models.wrap_angle(y - ct.h(m)), atol=5e-3)
        assert np.all(np.abs(r) < 0.1)


# ----- further sigma-point rules (unscented, Gauss-Hermite) ---------------
from paper_2207_00426_gb300 import workloads as W


def _mn(seed):
    rng = np.random.default_rng(seed)
    m = rng.standard_normal(5) * 0.5
    N = np.tril(0.2 * rng.standard_normal((5, 5))) + np.diag(rng.uniform(0.2, 0.5, 5))
    return m, N


@pytest.mark.parametrize("rule", ["cubature", "unscented", "gauss-hermite"])
def test_sigma_rules_match_the_first_two_moments(rule):
    m, N = _mn(1)
    X, w = slr.SIGMA_RULES[rule](m, N)
    assert np.all(w > 0) and abs(w.sum() - 1) < 1e-14
    np.testing.assert_allclose((w[:, None] * X).sum(0), m, atol=1e-14)
    C = sum(w[i] * np.outer(X[i] - m, X[i] - m) for i in range(len(w)))
    np.testing.assert_allclose(C, N @ N.T, atol=1e-14)


def test_gauss_hermite_is_exact_to_degree_five():
    # E over N(m, P) of x_1^4 and x_1^4 x_2 in closed form
    m, N = _mn(2)
    P = N @ N.T
    X, w = slr.gauss_hermite_points(m, N)
    e4 = 3 * P[0, 0] ** 2 + 6 * P[0, 0] * m[0] ** 2 + m[0] ** 4
    assert abs((w * X[:, 0] ** 4).sum() - e4) < 1e-13
    # x1^4 x2: E = m2 E[x1^4] + 4 P12 E[x1^3 centered moments] via Stein's lemma:
    # E[x1^4 x2] = m2 E[x1^4] + P12 E[4 x1^3] and E[x1^3] = m1^3 + 3 m1 P11
    e = m[1] * e4 + P[0, 1] * 4 * (m[0] ** 3 + 3 * m[0] * P[0, 0])
    assert abs((w * X[:, 0] ** 4 * X[:, 1]).sum() - e) < 1e-13
    # the third-degree rules are not exact for x^4
    Xc, wc = slr.cubature_points(m, N)
    assert abs((wc * Xc[:, 0] ** 4).sum() - e4) > 1e-3


@pytest.mark.parametrize("rule", ["unscented", "gauss-hermite"])
def test_sigma_rules_exact_on_linear_functions(rule):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((5, 5))
    u = rng.standard_normal(5)
    SQ = np.tril(rng.standard_normal((5, 5))) * 0.1 + np.eye(5) * 0.3

    class Lin:
        def f(self, x):
            return A @ x + u

        def SQ(self):
            return SQ

    m, N = _mn(4)
    F, c, S = slr.transition_sigma(Lin(), m, N, rule)
    np.testing.assert_allclose(F, A, atol=1e-12)
    np.testing.assert_allclose(c, u, atol=1e-12)
    np.testing.assert_allclose(S @ S.T, SQ @ SQ.T, atol=1e-12)


@pytest.mark.parametrize("rule", ["unscented", "gauss-hermite"])
def test_sigma_rules_ct_downdate_equals_residual_form(rule):
    d = W.ct_sequence(n=3, seed=5)
    ct = models.CTBearings(d["theta"], dt=d["dt"])
    m, N = _mn(6)
    m = d["x"][1] + 0.05 * m
    F, c, S = slr.transition_sigma(ct, m, N, rule)
    X, w = slr.SIGMA_RULES[rule](m, N)
    Zs = np.array([ct.f(x) for x in X])
    zbar = (w[:, None] * Zs).sum(0)
    Lam = ct.SQ() @ ct.SQ().T + sum(w[i] * np.outer(Zs[i] - zbar - F @ (X[i] - m),
                                                    Zs[i] - zbar - F @ (X[i] - m))
                                    for i in range(len(w)))
    np.testing.assert_allclose(S @ S.T, Lam, atol=1e-12)


# ----- Ricker / Poisson model: state-dependent observation noise ----------

def test_ricker_jacobians_match_central_differences():
    mdl = models.RickerPoisson(W.RICKER_THETA_TRUE)
    for x0 in (-1.0, 0.5, 2.0):
        x = np.array([x0])
        h = 1e-6
        df = (mdl.f(x + h) - mdl.f(x - h)) / (2 * h)
        dh = (mdl.h(x + h) - mdl.h(x - h)) / (2 * h)
        np.testing.assert_allclose(mdl.jac_f(x)[0, 0], df[0], rtol=1e-8)
        np.testing.assert_allclose(mdl.jac_h(x)[0, 0], dh[0], rtol=1e-8)


class _QuadraticObs:
    """y | x with E[y|x] = x^2 and Var[y|x] = x^2 + 1 (n_x = n_y = 1)."""
    nx = ny = 1

    def h(self, x):
        return x ** 2

    def cond_SR(self, x):
        return np.array([[np.sqrt(x[0] ** 2 + 1.0)]])

    def branch(self, z, ref):
        return z


def test_per_point_conditional_covariance_closed_form():
    # x ~ N(m, P): H = 2m, d = P - m^2, and Omega = E[Var(y|x)] + Var(E[y|x])
    # - H P H = m^2 + P + 1 + 2 P^2; Gauss-Hermite is exact to degree five
    m, P = 0.7, 0.3
    H, d, S = slr.observation_sigma(_QuadraticObs(), np.array([m]), np.array([[np.sqrt(P)]]),
                                    np.array([0.0]), "gauss-hermite")
    np.testing.assert_allclose(H[0, 0], 2 * m, rtol=1e-13)
    np.testing.assert_allclose(d[0], P - m * m, atol=1e-13)
    np.testing.assert_allclose(S[0, 0] ** 2, m * m + P + 1 + 2 * P * P, rtol=1e-13)


def test_per_point_factor_list_equals_constant_factor():
    m, N = _mn(7)
    d = W.ct_sequence(n=3, seed=8)
    ct = models.CTBearings(d["theta"], dt=d["dt"])
    X, w = slr.cubature_points(m, N)
    Zs = np.array([ct.f(x) for x in X])
    a = slr._gslr_sigma(m, N, Zs, w, ct.SQ())
    b = slr._gslr_sigma(m, N, Zs, w, [ct.SQ()] * len(w))
    for u, v in zip(a, b):
        np.testing.assert_allclose(u, v, atol=1e-15)


def test_point_mass_limit_is_taylor():
    mdl = models.RickerPoisson(W.RICKER_THETA_TRUE)
    m = np.array([1.2])
    for N, tol in ((np.zeros((1, 1)), 0.0), (np.array([[1e-6]]), 1e-9)):
        F, c, SQ = slr.transition_cubature(mdl, m, N)
        Ft, ct_, SQt = slr.transition_taylor(mdl, m)
        np.testing.assert_allclose(F, Ft, atol=tol, rtol=tol)
        np.testing.assert_allclose(c, ct_, atol=tol * 10)
        H, dd, SR = slr.observation_cubature(mdl, m, N, np.array([3.0]))
        Ht, dt_, SRt = slr.observation_taylor(mdl, m, np.array([3.0]))
        np.testing.assert_allclose(H, Ht, rtol=max(tol, 1e-15))
        np.testing.assert_allclose(SR, SRt, rtol=max(tol, 1e-15))


@pytest.mark.parametrize("m", [-0.5, 0.3, 1.2])
@pytest.mark.parametrize("P", [1e-3, 1e-2])
def test_ricker_gauss_hermite_slr_against_lognormal_moments(m, P):
    """x ~ N(m, P): the Poisson count y | x ~ Poisson(b e^x) has E[y] =
    b e^{m+P/2}, Cov(x, y) = P E[y] (Stein's lemma), Var(y) = E[y] +
    b^2 e^{2m+P}(e^P - 1), so H = E[y] and the residual Omega - E[y] =
    b^2 e^{2m+P}(e^P - 1 - P); the transition log a + x - e^x has F = 1 -
    e^{m+P/2} and Lambda - Q = e^{2m+P}(e^P - 1 - P).  The three-point
    Gauss-Hermite rule is exact to degree five and gives E[z^6] = 9 instead
    of 15, which fixes its leading errors: -P^2/20 (relative) in the
    regression slope, -5P/6 (relative) in the residual variances, -P^3/120
    (relative) in E[e^x]."""
    mdl = models.RickerPoisson(W.RICKER_THETA_TRUE)
    a, b, q = mdl.a, mdl.b, mdl.q
    N = np.array([[np.sqrt(P)]])
    H, d, S = slr.observation_sigma(mdl, np.array([m]), N, np.array([3.0]), "gauss-hermite")
    Ey = b * np.exp(m + P / 2)
    resid = np.exp(2 * m + P) * (np.exp(P) - 1 - P)
    assert abs(H[0, 0] / Ey - 1 + P * P / 20) <= P ** 3
    assert abs((d[0] + H[0, 0] * m) / Ey - 1) <= P ** 3
    # Omega = E[Var(y|x)] + residual of E[y|x]; the rule's E[b e^x] is
    # E[y] (1 - P^3/120), its residual b^2 resid (1 - 5P/6)
    assert abs((S[0, 0] ** 2 - Ey * (1 - P ** 3 / 120)) / (b * b * resid) - 1 + 5 * P / 6) <= 2 * P * P
    F, c, SQ = slr.transition_sigma(mdl, np.array([m]), N, "gauss-hermite")
    e = np.exp(m + P / 2)
    assert abs(F[0, 0] - (1 - e) - e * P * P / 20) <= e * P ** 3
    assert abs(c[0] + F[0, 0] * m - (np.log(a) + m - e)) <= e * P ** 3
    assert abs((SQ[0, 0] ** 2 - q) / resid - 1 + 5 * P / 6) <= 2 * P * P


@pytest.mark.parametrize("rule,z4", [("cubature", 1.0), ("unscented", 2.0)])
@pytest.mark.parametrize("m,P", [(1.2, 1e-2), (0.3, 1e-2), (-0.5, 1e-3)])
def test_degree_three_rules_against_lognormal_moments(rule, z4, m, P):
    """At n_x = 1 the cubature points m +- N (weights 1/2) and the unscented
    points m, m +- sqrt(2) N (weights 1/2, 1/4, kappa = 1) are exact to
    degree three and give E[z^4] = 1 and 2 instead of 3, so on the Poisson
    count of the Ricker model (E[y] = b e^{m+P/2} = H) the slope is off by
    (E[z^4] - 3) P/6 and the mean by (E[z^4] - 3) P^2/24 (relative)."""
    mdl = models.RickerPoisson(W.RICKER_THETA_TRUE)
    H, d, _ = slr.observation_sigma(mdl, np.array([m]), np.array([[np.sqrt(P)]]),
                                    np.array([3.0]), rule)
    Ey = mdl.b * np.exp(m + P / 2)
    assert abs(H[0, 0] / Ey - 1 - (z4 - 3) * P / 6) <= P * P
    assert abs((d[0] + H[0, 0] * m) / Ey - 1 - (z4 - 3) * P * P / 24) <= P ** 3
