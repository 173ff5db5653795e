"""Scan elements and associative operators of Sec. 3 (Lemmas 1-4, Tables 1-5),
square-root and standard (covariance) columns, and three scan orders.

Oracle: test infrastructure only.

Readings of the paper taken here (each also listed in the design notes):
* Table 2, b_k: the printed "d_{k-1}" is read as d_k, because y_k depends on
  d_k only (eq. linear-model) and eta_k in the same table uses d_k.
* Tables 1-2, standard eta_k: the printed (H F)^T S^{-1} H (y - H c - d) has a
  superfluous H (dimensions do not agree); it is read as
  (H F)^T S^{-1} (y - H c - d), which is what the square-root column gives.
* Lemma 2: the operand "J_k" / "Z_k" of the right element is read as J_j / Z_j.
* Table 4, standard E_k: "P_k ... Lambda_{k-1}" is read as P^f_k and Lambda_k.
* Alg. 2: n+1 smoothing elements k = 0 .. n, reverse scan, outputs k = 0 .. n.
* Z_k is made square as in the proof of Lemma 1: zero columns appended when
  n_x > n_y, Tria(Z_k) when n_x < n_y.

Filter element: tuple (A, b, U, eta, Z) (sqrt) or (A, b, C, eta, J) (standard).
Smoother element: (E, g, D) (sqrt) or (E, g, L) (standard).
"""
import numpy as np

from .linalg import tria, solve_lower, solve_upper


def _square_Z(Z, nx):
    """Make Z_k square as in the proof of Lemma 1."""
    ny = Z.shape[1]
    if ny < nx:
        return np.hstack([Z, np.zeros((nx, nx - ny))])
    if ny > nx:
        return tria(Z)
    return Z


# --------------------------------------------------------------------------
# Filter elements (Lemma 1)
# --------------------------------------------------------------------------
def sqrt_filter_element_first(F0, c0, SQ0, H1, d1, SR1, y1, m0, N0):
    """Table 1, right column (k = 1)."""
    nx = m0.shape[0]
    ny = y1.shape[0]
    m_pred = F0 @ m0 + c0
    N_pred = tria(np.hstack([F0 @ N0, SQ0]))
    Psi = tria(np.vstack([np.hstack([H1 @ N_pred, SR1]),
                          np.hstack([N_pred, np.zeros((nx, ny))])]))
    Y = Psi[:ny, :ny]
    K = solve_upper(Y.T, Psi[ny:, :ny].T).T            # K = Psi21 Psi11^{-1}
    A = np.zeros((nx, nx))
    b = m_pred + K @ (y1 - H1 @ m_pred - d1)
    U = Psi[ny:, ny:]
    Zr = solve_lower(Y, H1 @ F0).T                      # F0^T H1^T Y^{-T}
    eta = Zr @ solve_lower(Y, y1 - H1 @ c0 - d1)        # Z Y^{-1} (y - H c - d)
    return A, b, U, eta, _square_Z(Zr, nx)


def sqrt_filter_element(Fp, cp, SQp, H, d, SR, y):
    """Table 2, right column (1 < k <= n), with eq. sqrt-filter-init-2:
    Psi = Tria([[H S_Lambda_{k-1}, S_Omega_k], [S_Lambda_{k-1}, 0]])."""
    nx = Fp.shape[0]
    ny = y.shape[0]
    Psi = tria(np.vstack([np.hstack([H @ SQp, SR]),
                          np.hstack([SQp, np.zeros((nx, ny))])]))
    Y = Psi[:ny, :ny]
    K = solve_upper(Y.T, Psi[ny:, :ny].T).T
    A = (np.eye(nx) - K @ H) @ Fp
    b = cp + K @ (y - H @ cp - d)
    U = Psi[ny:, ny:]
    Zr = solve_lower(Y, H @ Fp).T
    eta = Zr @ solve_lower(Y, y - H @ cp - d)
    return A, b, U, eta, _square_Z(Zr, nx)


def std_filter_element_first(F0, c0, Q0, H1, d1, R1, y1, m0, P0):
    """Table 1, left column (k = 1); eta read without the extra H."""
    nx = m0.shape[0]
    m_pred = F0 @ m0 + c0
    P_pred = F0 @ P0 @ F0.T + Q0
    S = H1 @ P_pred @ H1.T + R1
    K = np.linalg.solve(S, H1 @ P_pred).T
    A = np.zeros((nx, nx))
    b = m_pred + K @ (y1 - H1 @ m_pred - d1)
    C = P_pred - K @ S @ K.T
    HF = H1 @ F0
    J = HF.T @ np.linalg.solve(S, HF)
    eta = HF.T @ np.linalg.solve(S, y1 - H1 @ c0 - d1)
    return A, b, C, eta, J


def std_filter_element(Fp, cp, Qp, H, d, R, y):
    """Table 2, left column (1 < k <= n); b uses d_k, eta without extra H."""
    nx = Fp.shape[0]
    S = H @ Qp @ H.T + R
    K = np.linalg.solve(S, H @ Qp).T
    A = (np.eye(nx) - K @ H) @ Fp
    b = cp + K @ (y - H @ cp - d)
    C = (np.eye(nx) - K @ H) @ Qp
    HF = H @ Fp
    J = HF.T @ np.linalg.solve(S, HF)
    eta = HF.T @ np.linalg.solve(S, y - H @ cp - d)
    return A, b, C, eta, J


# --------------------------------------------------------------------------
# Filter operator (Lemma 2, Table 3)
# --------------------------------------------------------------------------
def sqrt_filter_combine(ei, ej):
    """Table 3, right column, with Xi from eq. sqrt-filter-com-2."""
    Ai, bi, Ui, etai, Zi = ei
    Aj, bj, Uj, etaj, Zj = ej
    nx = Ai.shape[0]
    I = np.eye(nx)
    Xi = tria(np.vstack([np.hstack([Ui.T @ Zj, I]),
                         np.hstack([Zj, np.zeros((nx, nx))])]))
    X11 = Xi[:nx, :nx]
    X21 = Xi[nx:, :nx]
    X22 = Xi[nx:, nx:]
    T = solve_upper(X11.T, X21.T)                       # Xi11^{-T} Xi21^T
    Minv = I - Ui @ T                                   # (I + C_i J_j)^{-1}
    Aij = Aj @ Ai - Aj @ Ui @ T @ Ai
    bij = Aj @ Minv @ (bi + Ui @ (Ui.T @ etaj)) + bj
    V = solve_lower(X11, (Aj @ Ui).T).T                 # A_j U_i Xi11^{-T}
    Uij = tria(np.hstack([V, Uj]))
    etaij = Ai.T @ Minv.T @ (etaj - Zj @ (Zj.T @ bi)) + etai
    Zij = tria(np.hstack([Ai.T @ X22, Zi]))
    return Aij, bij, Uij, etaij, Zij


def std_filter_combine(ei, ej):
    """Table 3, left column (Saerkkae & Garcia-Fernandez, Lemma 8)."""
    Ai, bi, Ci, etai, Ji = ei
    Aj, bj, Cj, etaj, Jj = ej
    nx = Ai.shape[0]
    I = np.eye(nx)
    M = np.linalg.inv(I + Ci @ Jj)
    Mt = np.linalg.inv(I + Jj @ Ci)
    Aij = Aj @ M @ Ai
    bij = Aj @ M @ (bi + Ci @ etaj) + bj
    Cij = Aj @ M @ Ci @ Aj.T + Cj
    etaij = Ai.T @ Mt @ (etaj - Jj @ bi) + etai
    Jij = Ai.T @ Mt @ Jj @ Ai + Ji
    return Aij, bij, Cij, etaij, Jij


# --------------------------------------------------------------------------
# Smoother elements and operator (Lemmas 3-4, Tables 4-5)
# --------------------------------------------------------------------------
def sqrt_smoother_element(F, c, SQ, mf, Nf):
    """Table 4, right column (0 <= k < n), Phi from eq. smooth-init-2."""
    nx = mf.shape[0]
    Phi = tria(np.vstack([np.hstack([F @ Nf, SQ]),
                          np.hstack([Nf, np.zeros((nx, nx))])]))
    E = solve_upper(Phi[:nx, :nx].T, Phi[nx:, :nx].T).T  # Phi21 Phi11^{-1}
    g = mf - E @ (F @ mf + c)
    D = Phi[nx:, nx:]
    return E, g, D


def sqrt_smoother_element_last(mf, Nf):
    """Caption of Table 4: E_n = 0, g_n = m^f_n, D_n = N^f_n."""
    nx = mf.shape[0]
    return np.zeros((nx, nx)), mf.copy(), Nf.copy()


def std_smoother_element(F, c, Q, mf, Pf):
    """Table 4, left column (read with P^f_k and Lambda_k)."""
    E = np.linalg.solve(F @ Pf @ F.T + Q, F @ Pf).T
    g = mf - E @ (F @ mf + c)
    L = Pf - E @ F @ Pf
    return E, g, L


def sqrt_smoother_combine(ei, ej):
    """Table 5, right column."""
    Ei, gi, Di = ei
    Ej, gj, Dj = ej
    return Ei @ Ej, Ei @ gj + gi, tria(np.hstack([Ei @ Dj, Di]))


def std_smoother_combine(ei, ej):
    """Table 5, left column."""
    Ei, gi, Li = ei
    Ej, gj, Lj = ej
    return Ei @ Ej, Ei @ gj + gi, Ei @ Lj @ Ei.T + Li


# --------------------------------------------------------------------------
# Scan orders (Sec. 2.1, Alg. 1, Alg. 2)
# --------------------------------------------------------------------------
def scan_sequential(op, elems):
    """Inclusive prefix scan, left to right: out_k = a_1 x ... x a_k."""
    out = [elems[0]]
    for e in elems[1:]:
        out.append(op(out[-1], e))
    return out


def scan_tree(op, elems):
    """Inclusive prefix scan in the recursive pairwise order of the
    work-efficient (Blelloch / Ladner-Fischer) parallel scan: combine
    neighbours pairwise, scan the pairs recursively, then fill in the
    even positions.  Same result as scan_sequential for an associative op,
    different bracketing."""
    n = len(elems)
    if n == 1:
        return [elems[0]]
    pairs = [op(elems[2 * i], elems[2 * i + 1]) for i in range(n // 2)]
    if n % 2:
        pairs.append(elems[-1])
    P = scan_tree(op, pairs)
    out = [None] * n
    out[0] = elems[0]
    for i in range(n // 2):
        out[2 * i + 1] = P[i]
    for i in range(1, (n + 1) // 2):
        out[2 * i] = op(P[i - 1], elems[2 * i])
    return out


def scan_chunked(op, elems, bounds):
    """Inclusive prefix scan in reduce-then-scan order: chunks
    [bounds[i], bounds[i+1]) are folded to aggregates, the aggregates are
    scanned sequentially, and each chunk is re-scanned from its carry."""
    aggs = []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        a = elems[lo]
        for e in elems[lo + 1:hi]:
            a = op(a, e)
        aggs.append(a)
    out = []
    carry = None
    for (lo, hi), agg in zip(zip(bounds[:-1], bounds[1:]), aggs):
        acc = carry
        for e in elems[lo:hi]:
            acc = e if acc is None else op(acc, e)
            out.append(acc)
        carry = agg if carry is None else op(carry, agg)
    return out


def reverse_scan(scan, op, elems, *args):
    """Reverse (suffix) scan out_k = a_k x ... x a_n using a prefix-scan
    order on the reversed sequence with the operands swapped."""
    rop = lambda x, y: op(y, x)
    return scan(rop, elems[::-1], *args)[::-1]


# --------------------------------------------------------------------------
# Algorithms 1 and 2
# --------------------------------------------------------------------------
def parallel_sqrt_filter(F, c, SQ, H, d, SR, y, m0, N0, scan=scan_tree, *args):
    """Alg. 1 (square-root): elements by Lemma 1, scan with Table 3,
    m^f_{1:n} = b, N^f_{1:n} = U, m^f_0 = m0, N^f_0 = N0."""
    n = y.shape[0]
    elems = [sqrt_filter_element_first(F[0], c[0], SQ[0], H[0], d[0], SR[0],
                                       y[0], m0, N0)]
    for t in range(1, n):
        elems.append(sqrt_filter_element(F[t], c[t], SQ[t], H[t], d[t],
                                         SR[t], y[t]))
    pref = scan(sqrt_filter_combine, elems, *args)
    mf = np.vstack([m0[None]] + [p[1][None] for p in pref])
    Nf = np.stack([N0] + [p[2] for p in pref])
    return mf, Nf


def parallel_sqrt_smoother(F, c, SQ, mf, Nf, scan=scan_tree, *args):
    """Alg. 2 (square-root): elements k = 0..n by Lemma 3, reverse scan with
    Table 5, m^s = g, N^s = D."""
    n = F.shape[0]
    elems = [sqrt_smoother_element(F[k], c[k], SQ[k], mf[k], Nf[k])
             for k in range(n)]
    elems.append(sqrt_smoother_element_last(mf[n], Nf[n]))
    suf = reverse_scan(scan, sqrt_smoother_combine, elems, *args)
    return (np.stack([s[1] for s in suf]), np.stack([s[2] for s in suf]))


def parallel_std_filter(F, c, Q, H, d, R, y, m0, P0, scan=scan_tree, *args):
    """Alg. 1 (standard): elements by Tables 1-2 left, scan with Table 3 left."""
    n = y.shape[0]
    elems = [std_filter_element_first(F[0], c[0], Q[0], H[0], d[0], R[0],
                                      y[0], m0, P0)]
    for t in range(1, n):
        elems.append(std_filter_element(F[t], c[t], Q[t], H[t], d[t], R[t],
                                        y[t]))
    pref = scan(std_filter_combine, elems, *args)
    mf = np.vstack([m0[None]] + [p[1][None] for p in pref])
    Pf = np.stack([P0] + [p[2] for p in pref])
    return mf, Pf


def parallel_std_smoother(F, c, Q, mf, Pf, scan=scan_tree, *args):
    """Alg. 2 (standard): Table 4 left elements, Table 5 left operator."""
    n = F.shape[0]
    elems = [std_smoother_element(F[k], c[k], Q[k], mf[k], Pf[k])
             for k in range(n)]
    elems.append((np.zeros_like(F[0]), mf[n].copy(), Pf[n].copy()))
    suf = reverse_scan(scan, std_smoother_combine, elems, *args)
    return (np.stack([s[1] for s in suf]), np.stack([s[2] for s in suf]))
