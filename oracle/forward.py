"""Forward-mode (tangent) derivative of the pseudo log-likelihood through
the fixed point of Alg. 3 -- the second gradient route of this oracle, next
to the central differences of ipls.nll_grad_fd.  Oracle: test
infrastructure only; FP64, sequential, plain NumPy.

Every quantity x of the sequential smoother is carried with its tangent
dx = sum_j (d x / d theta_j) e_j, stored as a trailing axis of length P (one
slot per parameter), and each step applies the product rule to the
formulas the sequential oracle evaluates:

* cubature SLR (Sec. 4.3): sigma points X_i = m +- sqrt(n_x) N e_i,
  Z_i = f(X_i) with dZ_i = J_f(X_i) dX_i, the regression matrix
  G = Cross (N N^T)^{-1}, the offset z_bar - G m, and the noise factor as
  the Tria of the residual columns (equal in product to the DownDate form
  of eqs. lambda-prime and sqr-lambda-sigma-point);
* the square-root Kalman filter step and the RTS step of kalman.py, with
  the pseudo log-likelihood terms of Sec. 5.1;
* Tria (Sec. 2.2): with A of full row rank, L = Tria(A) is the Cholesky
  factor of C = A A^T, so dL = L Phi(L^{-1} dC L^{-T}) with
  dC = dA A^T + A dA^T and Phi(X) the lower triangle of X with its diagonal
  halved (the derivative of the Cholesky factorisation).  Every Tria of the
  sequential smoother has full row rank (its blocks hold S_Lambda, S_Omega
  or a filtering factor).

Alg. 3 is iterated with the tangents of the trajectory until both the
trajectory and its tangent have settled; the tangent of the pseudo
log-likelihood is then its total derivative through the fixed point (the
tangent iteration is the linearised fixed-point map, whose limit is the
solution of eq. implicity_function_theorem).  The model supplies f, h,
their Jacobians, SQ, SR, branch and the parameter derivatives dSQ_dtheta,
dSR_dtheta (arrays with the trailing parameter axis).
"""
import numpy as np

from .kalman import LOG2PI
from .linalg import tria


def _mm(A, dA, B, dB):
    """(A B, dA B + A dB) for matrices (or matrix-vector products)."""
    val = A @ B
    if B.ndim == 1:
        tan = np.einsum("ijp,j->ip", dA, B) + np.einsum("ij,jp->ip", A, dB)
    else:
        tan = np.einsum("ijp,jk->ikp", dA, B) + np.einsum("ij,jkp->ikp", A, dB)
    return val, tan


def _const(A, P):
    return np.zeros(A.shape + (P,))


def tria_jvp(A, dA):
    """(Tria(A), its tangent) for A (n x m) of full row rank."""
    L = tria(A)
    dC = np.einsum("ikp,jk->ijp", dA, A)
    dC = dC + np.swapaxes(dC, 0, 1)
    Li = np.linalg.inv(L)
    X = np.einsum("ik,klp,jl->ijp", Li, dC, Li)
    n = L.shape[0]
    low = np.tril(np.ones((n, n))) - 0.5 * np.eye(n)
    return L, np.einsum("ik,kjp->ijp", L, X * low[:, :, None])


def _solve_right(B, dB, Y, dY):
    """(X, dX) with X Y = B for invertible Y: dX = (dB - X dY) Y^{-1}."""
    Yi = np.linalg.inv(Y)
    X = B @ Yi
    dX = np.einsum("ikp,kj->ijp", dB - np.einsum("ik,kjp->ijp", X, dY), Yi)
    return X, dX


def _gslr_cubature(m, dm, N, dN, fun, jac, S, dS):
    """Cubature regression of z = fun(x) about (m, N) with additive noise
    factor S: (G, off, L) and tangents (Sec. 4.3, residual form)."""
    nx = m.shape[0]
    P = dm.shape[-1]
    s = np.sqrt(nx)
    X, dX = [], []
    for sgn in (1.0, -1.0):
        for i in range(nx):
            X.append(m + sgn * s * N[:, i])
            dX.append(dm + sgn * s * dN[:, i, :])
    w = 1.0 / (2 * nx)
    Z = [fun(x) for x in X]
    dZ = [jac(x) @ dx for x, dx in zip(X, dX)]
    zbar = w * np.sum(Z, axis=0)
    dzbar = w * np.sum(dZ, axis=0)
    Cross = sum(w * np.outer(Z[i] - zbar, X[i] - m) for i in range(2 * nx))
    dCross = sum(w * (np.einsum("ip,j->ijp", dZ[i] - dzbar, X[i] - m)
                      + np.einsum("i,jp->ijp", Z[i] - zbar, dX[i] - dm)) for i in range(2 * nx))
    Pm, dPm = _mm(N, dN, N.T, np.swapaxes(dN, 0, 1))
    G, dG = _solve_right(Cross, dCross, Pm, dPm)
    off = zbar - G @ m
    doff = dzbar - np.einsum("ijp,j->ip", dG, m) - G @ dm
    ny = zbar.shape[0]
    cols, dcols = [], []
    for i in range(2 * nx):
        cols.append(np.sqrt(w) * S)
        dcols.append(np.sqrt(w) * dS)
    for i in range(2 * nx):
        r = Z[i] - zbar - G @ (X[i] - m)
        dr = (dZ[i] - dzbar - np.einsum("ijp,j->ip", dG, X[i] - m) - G @ (dX[i] - dm))
        cols.append(np.sqrt(w) * r[:, None])
        dcols.append(np.sqrt(w) * dr[:, None, :])
    L, dL = tria_jvp(np.hstack(cols), np.concatenate(dcols, axis=1))
    assert L.shape == (ny, ny) and dL.shape == (ny, ny, P)
    return G, dG, off, doff, L, dL


def linearize_jvp(model, ms, dms, Ns, dNs, y):
    """Gamma^sqrt (eq. Gamma-s) with the cubature rule for every step and its
    tangent: transition t about row t, observation of x_{t+1} about row
    t + 1 (bearings on the branch nearest h(m), as slr.observation_cubature)."""
    n = y.shape[0]
    dSQ, dSR = model.dSQ_dtheta(), model.dSR_dtheta()
    SQ, SR = model.SQ(), model.SR()
    out = []
    for t in range(n):
        F, dF, c, dc, L, dL = _gslr_cubature(ms[t], dms[t], Ns[t], dNs[t], model.f, model.jac_f,
                                             SQ, dSQ)
        ref = model.h(ms[t + 1])
        H, dH, d, dd, R, dR = _gslr_cubature(ms[t + 1], dms[t + 1], Ns[t + 1], dNs[t + 1],
                                             lambda x: model.branch(model.h(x), ref),
                                             model.jac_h, SR, dSR)
        d = d + (y[t] - model.branch(y[t], ref))
        out.append((F, dF, c, dc, L, dL, H, dH, d, dd, R, dR))
    return out


def sqrt_filter_jvp(G, y, m0, N0, P):
    """Sequential square-root Kalman filter (kalman.sqrt_filter) with
    tangents; the prior (m0, N0) does not depend on theta.  Returns mf, dmf,
    Nf, dNf, the pseudo log-likelihood and its tangent (P,)."""
    n, ny = y.shape
    nx = m0.shape[0]
    mf = np.zeros((n + 1, nx)); dmf = np.zeros((n + 1, nx, P))
    Nf = np.zeros((n + 1, nx, nx)); dNf = np.zeros((n + 1, nx, nx, P))
    mf[0], Nf[0] = m0, N0
    ell, dell = 0.0, np.zeros(P)
    for t in range(n):
        F, dF, c, dc, SQ, dSQ, H, dH, d, dd, SR, dSR = G[t]
        mp, dmp = _mm(F, dF, mf[t], dmf[t])
        mp, dmp = mp + c, dmp + dc
        FN, dFN = _mm(F, dF, Nf[t], dNf[t])
        Np, dNp = tria_jvp(np.hstack([FN, SQ]), np.concatenate([dFN, dSQ], axis=1))
        HN, dHN = _mm(H, dH, Np, dNp)
        A = np.vstack([np.hstack([HN, SR]), np.hstack([Np, np.zeros((nx, ny))])])
        dA = np.concatenate([np.concatenate([dHN, dSR], axis=1),
                             np.concatenate([dNp, np.zeros((nx, ny, P))], axis=1)], axis=0)
        Psi, dPsi = tria_jvp(A, dA)
        Y, dY = Psi[:ny, :ny], dPsi[:ny, :ny]
        K, dK = _solve_right(Psi[ny:, :ny], dPsi[ny:, :ny], Y, dY)
        Hm, dHm = _mm(H, dH, mp, dmp)
        v = y[t] - Hm - d
        dv = -dHm - dd
        mf[t + 1] = mp + K @ v
        dmf[t + 1] = dmp + np.einsum("ijp,j->ip", dK, v) + K @ dv
        Nf[t + 1], dNf[t + 1] = Psi[ny:, ny:], dPsi[ny:, ny:]
        Yi = np.linalg.inv(Y)
        e = Yi @ v
        de = Yi @ (dv - np.einsum("ijp,j->ip", dY, e))
        dg = np.diagonal(Y)
        ell += -0.5 * (ny * LOG2PI + 2.0 * np.sum(np.log(np.abs(dg))) + e @ e)
        dell += -(np.sum(np.diagonal(dY, axis1=0, axis2=1) / dg[None, :], axis=1) + e @ de)
    return mf, dmf, Nf, dNf, ell, dell


def sqrt_smoother_jvp(G, mf, dmf, Nf, dNf):
    """Sequential square-root RTS smoother (kalman.sqrt_smoother) with
    tangents."""
    n = len(G)
    nx = mf.shape[1]
    P = dmf.shape[-1]
    ms, dms = mf.copy(), dmf.copy()
    Ns, dNs = Nf.copy(), dNf.copy()
    Z = np.zeros((nx, nx))
    dZ = np.zeros((nx, nx, P))
    for k in range(n - 1, -1, -1):
        F, dF, c, dc, SQ, dSQ = G[k][:6]
        FN, dFN = _mm(F, dF, Nf[k], dNf[k])
        A = np.vstack([np.hstack([FN, SQ]), np.hstack([Nf[k], Z])])
        dA = np.concatenate([np.concatenate([dFN, dSQ], axis=1),
                             np.concatenate([dNf[k], dZ], axis=1)], axis=0)
        Phi, dPhi = tria_jvp(A, dA)
        E, dE = _solve_right(Phi[nx:, :nx], dPhi[nx:, :nx], Phi[:nx, :nx], dPhi[:nx, :nx])
        Fm, dFm = _mm(F, dF, mf[k], dmf[k])
        u, du = Fm + c, dFm + dc
        Eu, dEu = _mm(E, dE, u, du)
        g, dg = mf[k] - Eu, dmf[k] - dEu
        Em, dEm = _mm(E, dE, ms[k + 1], dms[k + 1])
        ms[k], dms[k] = Em + g, dEm + dg
        EN, dEN = _mm(E, dE, Ns[k + 1], dNs[k + 1])
        Ns[k], dNs[k] = tria_jvp(np.hstack([EN, Phi[nx:, nx:]]),
                                 np.concatenate([dEN, dPhi[nx:, nx:]], axis=1))
    return ms, dms, Ns, dNs


def nll_grad_forward(model, y, m0, N0, tol=1e-12, max_iters=200):
    """Negative pseudo log-likelihood at the fixed point of Alg. 3 (cubature,
    prior broadcast as the initial trajectory) and its total derivative in
    theta by forward mode.  Iterates until the trajectory and its tangent
    change by less than tol (max-norm) in one iteration.  Returns
    (nll, grad, iterations)."""
    n = y.shape[0]
    P = model.dSQ_dtheta().shape[-1]
    ms = np.tile(m0, (n + 1, 1))
    Ns = np.tile(N0, (n + 1, 1, 1))
    dms = np.zeros(ms.shape + (P,))
    dNs = np.zeros(Ns.shape + (P,))
    ell, dell = np.nan, np.full(P, np.nan)
    for it in range(1, max_iters + 1):
        G = linearize_jvp(model, ms, dms, Ns, dNs, y)
        mf, dmf, Nf, dNf, ell, dell = sqrt_filter_jvp(G, y, m0, N0, P)
        ms2, dms2, Ns2, dNs2 = sqrt_smoother_jvp(G, mf, dmf, Nf, dNf)
        delta = max(np.max(np.abs(ms2 - ms)), np.max(np.abs(dms2 - dms)))
        ms, dms, Ns, dNs = ms2, dms2, Ns2, dNs2
        if delta < tol:
            break
    return -ell, -dell, it
