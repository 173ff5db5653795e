"""Square-root statistical linear regression (Sec. 4).  Oracle: test
infrastructure only.

Cubature rule (Sec. 4.3 cites the cubature Kalman filter without printing the
rule; reading): the third-degree spherical-radial rule with 2 n_x points
X_i = m +- sqrt(n_x) N e_i and equal weights w^m = w^c = 1/(2 n_x).

The transition noise is additive, so the conditional square root
S_x[x_k | x_{k-1}](X_i) is the constant S_Q for every point.

Bearings are angles (model.branch): every transformed point and the
measurement are taken on the branch nearest h(m); the 2 pi multiple that
this moves y by is added to d, so that y - H x - d uses the wrapped residual.
"""
import numpy as np

from .linalg import tria, downdate, solve_lower, solve_upper


def cubature_points(m, N):
    """Sigma points and weights of the third-degree spherical-radial rule."""
    nx = m.shape[0]
    s = np.sqrt(nx)
    X = [m + s * N[:, i] for i in range(nx)] + [m - s * N[:, i] for i in range(nx)]
    w = np.full(2 * nx, 1.0 / (2 * nx))
    return np.array(X), w


# Further positive-weight sigma-point rules (Sec. 4.3 admits any rule with
# positive weights; readings: the unscented transform with alpha = 1,
# beta = 0, kappa = 1, and the three-point Gauss-Hermite rule per dimension).
UT_KAPPA = 1.0


def unscented_points(m, N, kappa=UT_KAPPA):
    """2 n_x + 1 points m, m +- sqrt(n_x + lambda) N e_i with lambda = kappa
    (alpha = 1) and weights lambda / (n_x + lambda), 1 / (2 (n_x + lambda));
    with beta = 0 the mean and covariance weights coincide."""
    nx = m.shape[0]
    lam = kappa
    s = np.sqrt(nx + lam)
    X = [m] + [m + s * N[:, i] for i in range(nx)] + [m - s * N[:, i] for i in range(nx)]
    w = np.array([lam / (nx + lam)] + [0.5 / (nx + lam)] * (2 * nx))
    return np.array(X), w


def gauss_hermite_points(m, N):
    """The tensor product of the three-point Gauss-Hermite rule for N(0, 1)
    (nodes 0, +-sqrt(3), weights 2/3, 1/6, 1/6): 3^n_x points m + N xi,
    weight prod_k w(xi_k)."""
    nx = m.shape[0]
    nodes = np.array([0.0, np.sqrt(3.0), -np.sqrt(3.0)])
    w1 = np.array([2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0])
    X, w = [], []
    for p in range(3 ** nx):
        digits = [(p // 3 ** k) % 3 for k in range(nx)]
        xi = nodes[digits]
        X.append(m + N @ xi)
        w.append(np.prod(w1[digits]))
    return np.array(X), np.array(w)


SIGMA_RULES = {"cubature": cubature_points, "unscented": unscented_points,
               "gauss-hermite": gauss_hermite_points}


def _gslr_sigma(m, N, Zs, w, S_cond, X=None):
    """Sec. 4.3: z_bar (eq. z-bar), the regression matrix
    sum_i w_i (Z_i - z_bar)(X_i - m)^T (N N^T)^{-1}, the offset
    z_bar - G m, and the noise factor
    DownDate(Tria(sqrt(w_1) S_1, ..., sqrt(w_s) S_s, Z), G N)
    (eqs. lambda-prime and sqr-lambda-sigma-point).  X: the points (default:
    the cubature rule's)."""
    if X is None:
        X, _ = cubature_points(m, N)
    zbar = np.sum(w[:, None] * Zs, axis=0)
    Cross = sum(w[i] * np.outer(Zs[i] - zbar, X[i] - m) for i in range(len(w)))
    # G = Cross (N N^T)^{-1} = ((N N^T)^{-1} Cross^T)^T via two triangular solves
    G = solve_upper(N.T, solve_lower(N, Cross.T)).T
    off = zbar - G @ m
    Zdev = np.array([np.sqrt(w[i]) * (Zs[i] - zbar) for i in range(len(w))]).T
    # S_cond: one conditional factor for every point, or a list of them
    S_i = S_cond if isinstance(S_cond, list) else [S_cond] * len(w)
    blocks = [np.sqrt(w[i]) * S_i[i] for i in range(len(w))] + [Zdev]
    S_prime = tria(np.hstack(blocks))
    S = downdate(S_prime, G @ N)
    return G, off, S


def residual_noise_factor(m, N, Zs, w, S_cond, G):
    """Cross-check of the DownDate result: Tria of
    [sqrt(w_i) S_i, sqrt(w_i) (Z_i - z_bar - G (X_i - m))]_i has the same
    product S S^T, because sum_i w_i (X_i - m)(X_i - m)^T = N N^T for this
    rule and G is the regression matrix."""
    X, _ = cubature_points(m, N)
    zbar = np.sum(w[:, None] * Zs, axis=0)
    cols = [np.sqrt(w[i]) * S_cond for i in range(len(w))]
    cols += [np.sqrt(w[i]) * (Zs[i] - zbar - G @ (X[i] - m))[:, None]
             for i in range(len(w))]
    return tria(np.hstack(cols))


def _point_mass(N):
    """A zero factor (a point-mass marginal, e.g. a known initial state):
    every sigma point is m and the regression is undefined; its limit as
    N -> 0 is the Taylor linearisation (Sec. 4.2), which is taken instead."""
    return np.min(np.abs(np.diag(N))) < 1e-300


def transition_cubature(model, m, N):
    """(F_{k-1}, c_{k-1}, S_Lambda_{k-1}) from (m^s_{k-1}, N^s_{k-1})."""
    if _point_mass(N):
        return transition_taylor(model, m)
    X, w = cubature_points(m, N)
    Zs = np.array([model.f(x) for x in X])
    return _gslr_sigma(m, N, Zs, w, model.SQ())


def _cond_factors(model, X):
    """Per-point conditional observation factors for a model whose noise
    depends on the state, else the constant S_R."""
    if hasattr(model, "cond_SR"):
        return [model.cond_SR(x) for x in X]
    return model.SR()


def observation_cubature(model, m, N, y):
    """(H_k, d_k, S_Omega_k) from (m^s_k, N^s_k); bearings on the branch
    nearest h(m), d absorbing the 2 pi shift of y."""
    if _point_mass(N):
        return observation_taylor(model, m, y)
    X, w = cubature_points(m, N)
    ref = model.h(m)
    Zs = np.array([model.branch(model.h(x), ref) for x in X])
    H, d, S = _gslr_sigma(m, N, Zs, w, _cond_factors(model, X))
    d = d + (y - model.branch(y, ref))
    return H, d, S


def transition_sigma(model, m, N, rule):
    """(F, c, S_Lambda) with the named sigma-point rule."""
    if _point_mass(N):
        return transition_taylor(model, m)
    X, w = SIGMA_RULES[rule](m, N)
    Zs = np.array([model.f(x) for x in X])
    return _gslr_sigma(m, N, Zs, w, model.SQ(), X)


def observation_sigma(model, m, N, y, rule):
    """(H, d, S_Omega) with the named sigma-point rule, bearings on the
    branch nearest h(m) as in observation_cubature."""
    if _point_mass(N):
        return observation_taylor(model, m, y)
    X, w = SIGMA_RULES[rule](m, N)
    ref = model.h(m)
    Zs = np.array([model.branch(model.h(x), ref) for x in X])
    H, d, S = _gslr_sigma(m, N, Zs, w, _cond_factors(model, X), X)
    return H, d + (y - model.branch(y, ref)), S


def transition_taylor(model, m):
    """Sec. 4.2: F = grad f(m^s_{k-1}), c = f(m) - F m, S_Lambda = S_Q."""
    F = model.jac_f(m)
    return F, model.f(m) - F @ m, model.SQ()


def observation_taylor(model, m, y):
    """Sec. 4.2: H = grad h(m^s_k), d = h(m) - H m (+ branch shift of y),
    S_Omega = S_R (the conditional factor at m for a state-dependent noise)."""
    H = model.jac_h(m)
    ref = model.h(m)
    d = ref - H @ m + (y - model.branch(y, ref))
    SR = model.cond_SR(m) if hasattr(model, "cond_SR") else model.SR()
    return H, d, SR


def linearize(model, ms, Ns, y, method):
    """Gamma^sqrt (eq. Gamma-s) for all steps: transition t from
    (ms[t], Ns[t]), observation of x_{t+1} from (ms[t+1], Ns[t+1])."""
    n = y.shape[0]
    nx, ny = model.nx, model.ny
    F = np.zeros((n, nx, nx)); c = np.zeros((n, nx)); SQ = np.zeros((n, nx, nx))
    H = np.zeros((n, ny, nx)); d = np.zeros((n, ny)); SR = np.zeros((n, ny, ny))
    for t in range(n):
        if method == "cubature":
            F[t], c[t], SQ[t] = transition_cubature(model, ms[t], Ns[t])
            H[t], d[t], SR[t] = observation_cubature(model, ms[t + 1], Ns[t + 1], y[t])
        elif method == "extended":
            F[t], c[t], SQ[t] = transition_taylor(model, ms[t])
            H[t], d[t], SR[t] = observation_taylor(model, ms[t + 1], y[t])
        elif method in SIGMA_RULES:
            F[t], c[t], SQ[t] = transition_sigma(model, ms[t], Ns[t], method)
            H[t], d[t], SR[t] = observation_sigma(model, ms[t + 1], Ns[t + 1], y[t], method)
        else:
            raise ValueError(method)
    return F, c, SQ, H, d, SR


# --------------------------------------------------------------------------
# Standard (covariance) form of the same regressions, for the standard
# parallel filter and smoother (left columns of Tables 1-5): Sec. 4.1's
# statistical linear regression written with covariances,
#   F = Psi^T P^{-1},  c = z_bar - F m,  Lambda = Phi - F P F^T + Q,
# Psi = sum_i w (X_i - m)(Z_i - z_bar)^T, Phi = sum_i w (Z_i - z_bar)(...)^T.
# --------------------------------------------------------------------------
def _gslr_cov(m, P, Zs, w, Q):
    N = np.linalg.cholesky(P)
    X, _ = cubature_points(m, N)
    zbar = np.sum(w[:, None] * Zs, axis=0)
    Psi = sum(w[i] * np.outer(X[i] - m, Zs[i] - zbar) for i in range(len(w)))
    Phi = sum(w[i] * np.outer(Zs[i] - zbar, Zs[i] - zbar) for i in range(len(w)))
    G = np.linalg.solve(P, Psi).T
    return G, zbar - G @ m, Phi - G @ P @ G.T + Q


def transition_cubature_std(model, m, P):
    """(F, c, Lambda) from (m^s_{k-1}, P^s_{k-1}), covariance form."""
    X, w = cubature_points(m, np.linalg.cholesky(P))
    Zs = np.array([model.f(x) for x in X])
    SQ = model.SQ()
    return _gslr_cov(m, P, Zs, w, SQ @ SQ.T)


def observation_cubature_std(model, m, P, y):
    """(H, d, Omega) from (m^s_k, P^s_k), covariance form, bearings on the
    branch nearest h(m) as in observation_cubature."""
    X, w = cubature_points(m, np.linalg.cholesky(P))
    ref = model.h(m)
    Zs = np.array([model.branch(model.h(x), ref) for x in X])
    SR = model.SR()
    H, d, R = _gslr_cov(m, P, Zs, w, SR @ SR.T)
    return H, d + (y - model.branch(y, ref)), R


def linearize_std(model, ms, Ps, y):
    """The covariance-form linearisation of every step (cubature):
    transition t from (ms[t], Ps[t]), observation from (ms[t+1], Ps[t+1])."""
    n = y.shape[0]
    nx, ny = model.nx, model.ny
    F = np.zeros((n, nx, nx)); c = np.zeros((n, nx)); Q = np.zeros((n, nx, nx))
    H = np.zeros((n, ny, nx)); d = np.zeros((n, ny)); R = np.zeros((n, ny, ny))
    for t in range(n):
        F[t], c[t], Q[t] = transition_cubature_std(model, ms[t], Ps[t])
        H[t], d[t], R[t] = observation_cubature_std(model, ms[t + 1], Ps[t + 1], y[t])
    return F, c, Q, H, d, R

