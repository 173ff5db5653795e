"""Pins of the scan elements and operators (Lemmas 1-4, Tables 1-5): every
scan order reproduces the sequential filter/smoother; the square-root and
standard columns agree through U U^T = C, Z Z^T = J, D D^T = L; the operator
is associative; the Xi identities of the proof of Lemma 2 hold."""
import numpy as np
import pytest

from oracle import parallel as P
from oracle.kalman import sqrt_filter, sqrt_smoother, cov_filter, cov_smoother
from paper_2207_00426_gb300.workloads import random_lgssm


def _model(n, nx, ny, seed):
    m = random_lgssm(n, nx, ny, seed=seed)
    m["Q"] = m["SQ"] @ np.transpose(m["SQ"], (0, 2, 1))
    m["R"] = m["SR"] @ np.transpose(m["SR"], (0, 2, 1))
    return m


def _args(m):
    return m["F"], m["c"], m["SQ"], m["H"], m["d"], m["SR"], m["y"], m["m0"], m["N0"]


def _gram(X):
    return X @ np.transpose(X, (0, 2, 1))


@pytest.mark.parametrize("order", ["sequential", "tree", "chunked"])
@pytest.mark.parametrize("nx,ny", [(4, 2), (5, 2), (1, 2), (3, 3)])
def test_parallel_sqrt_filter_smoother_equal_sequential(order, nx, ny):
    n = 23
    m = _model(n, nx, ny, seed=nx + 7 * ny)
    mf, Nf, _ = sqrt_filter(*_args(m))
    ms, Ns = sqrt_smoother(m["F"], m["c"], m["SQ"], mf, Nf)
    if order == "sequential":
        scan, extra = P.scan_sequential, ()
    elif order == "tree":
        scan, extra = P.scan_tree, ()
    else:
        scan, extra = P.scan_chunked, ([0, 3, 4, 11, 17, 23],)
    mf2, Nf2 = P.parallel_sqrt_filter(*_args(m), scan, *extra)
    np.testing.assert_allclose(mf2, mf, atol=1e-10)
    np.testing.assert_allclose(_gram(Nf2), _gram(Nf), atol=1e-10)
    if order == "chunked":
        extra = ([0, 5, 6, 13, 20, 24],)            # n + 1 smoothing elements
    ms2, Ns2 = P.parallel_sqrt_smoother(m["F"], m["c"], m["SQ"], mf, Nf, scan, *extra)
    np.testing.assert_allclose(ms2, ms, atol=1e-10)
    np.testing.assert_allclose(_gram(Ns2), _gram(Ns), atol=1e-10)


def test_parallel_standard_equal_covariance_filter():
    n = 19
    m = _model(n, 4, 2, seed=3)
    P0 = m["N0"] @ m["N0"].T
    mf, Pf, _, _ = cov_filter(m["F"], m["c"], m["Q"], m["H"], m["d"], m["R"], m["y"], m["m0"], P0)
    ms, Ps = cov_smoother(m["F"], m["c"], m["Q"], mf, Pf)
    mf2, Pf2 = P.parallel_std_filter(m["F"], m["c"], m["Q"], m["H"], m["d"], m["R"], m["y"], m["m0"], P0)
    ms2, Ps2 = P.parallel_std_smoother(m["F"], m["c"], m["Q"], mf, Pf)
    np.testing.assert_allclose(mf2, mf, atol=1e-10)
    np.testing.assert_allclose(Pf2, Pf, atol=1e-10)
    np.testing.assert_allclose(ms2, ms, atol=1e-10)
    np.testing.assert_allclose(Ps2, Ps, atol=1e-10)


def _elements(m):
    n = m["y"].shape[0]
    sq = [P.sqrt_filter_element_first(m["F"][0], m["c"][0], m["SQ"][0], m["H"][0], m["d"][0],
                                      m["SR"][0], m["y"][0], m["m0"], m["N0"])]
    st = [P.std_filter_element_first(m["F"][0], m["c"][0], m["Q"][0], m["H"][0], m["d"][0],
                                     m["R"][0], m["y"][0], m["m0"], m["N0"] @ m["N0"].T)]
    for t in range(1, n):
        sq.append(P.sqrt_filter_element(m["F"][t], m["c"][t], m["SQ"][t], m["H"][t], m["d"][t],
                                        m["SR"][t], m["y"][t]))
        st.append(P.std_filter_element(m["F"][t], m["c"][t], m["Q"][t], m["H"][t], m["d"][t],
                                       m["R"][t], m["y"][t]))
    return sq, st


def _assert_same(es, et, atol=1e-10):
    A, b, U, eta, Z = es
    A2, b2, C, eta2, J = et
    np.testing.assert_allclose(A, A2, atol=atol)
    np.testing.assert_allclose(b, b2, atol=atol)
    np.testing.assert_allclose(U @ U.T, C, atol=atol)
    np.testing.assert_allclose(eta, eta2, atol=atol)
    np.testing.assert_allclose(Z @ Z.T, J, atol=atol)


def test_sqrt_and_standard_elements_and_operator_agree():
    m = _model(6, 5, 2, seed=11)
    sq, st = _elements(m)
    for es, et in zip(sq, st):
        _assert_same(es, et)
    for i in range(5):
        _assert_same(P.sqrt_filter_combine(sq[i], sq[i + 1]),
                     P.std_filter_combine(st[i], st[i + 1]))
    # combine of aggregates (full-rank Z)
    a = P.sqrt_filter_combine(P.sqrt_filter_combine(sq[1], sq[2]), sq[3])
    b = P.sqrt_filter_combine(sq[4], P.sqrt_filter_combine(sq[5], sq[2]))
    a2 = P.std_filter_combine(P.std_filter_combine(st[1], st[2]), st[3])
    b2 = P.std_filter_combine(st[4], P.std_filter_combine(st[5], st[2]))
    _assert_same(P.sqrt_filter_combine(a, b), P.std_filter_combine(a2, b2), atol=1e-9)


def test_filter_operator_associative():
    m = _model(4, 5, 2, seed=12)
    sq, _ = _elements(m)
    a, b, c = sq[1], sq[2], sq[3]
    left = P.sqrt_filter_combine(P.sqrt_filter_combine(a, b), c)
    right = P.sqrt_filter_combine(a, P.sqrt_filter_combine(b, c))
    for x, y in zip(left, right):
        if x.ndim == 2:
            np.testing.assert_allclose(x @ x.T, y @ y.T, atol=1e-10)
        np.testing.assert_allclose(x if x.ndim == 1 else x @ x.T,
                                   y if y.ndim == 1 else y @ y.T, atol=1e-10)
    np.testing.assert_allclose(left[0], right[0], atol=1e-10)


def test_xi_identities_and_inverse():
    """Eq. Xis and eq. sqrt-filter-com-3 of the proof of Lemma 2."""
    from oracle.linalg import tria
    m = _model(3, 5, 2, seed=13)
    sq, st = _elements(m)
    Ui, Zj = sq[1][2], sq[2][4]
    Ci, Jj = Ui @ Ui.T, Zj @ Zj.T
    nx = 5
    Xi = tria(np.vstack([np.hstack([Ui.T @ Zj, np.eye(nx)]), np.hstack([Zj, np.zeros((nx, nx))])]))
    X11, X21, X22 = Xi[:nx, :nx], Xi[nx:, :nx], Xi[nx:, nx:]
    np.testing.assert_allclose(X11 @ X11.T, Ui.T @ Jj @ Ui + np.eye(nx), atol=1e-10)
    np.testing.assert_allclose(X21 @ X11.T, Jj @ Ui, atol=1e-10)
    np.testing.assert_allclose(X21 @ X21.T + X22 @ X22.T, Jj, atol=1e-10)
    lhs = np.linalg.inv(np.eye(nx) + Ci @ Jj)
    rhs = np.eye(nx) - Ui @ np.linalg.solve(X11.T, X21.T)
    np.testing.assert_allclose(lhs, rhs, atol=1e-10)


def test_first_element_Z_eta_do_not_matter():
    """A_1 = 0, so prefix b and U never use Z_1 and eta_1."""
    m = _model(9, 5, 2, seed=14)
    sq, _ = _elements(m)
    z = list(sq[0])
    z[3] = np.zeros_like(z[3]); z[4] = np.zeros_like(z[4])
    p1 = P.scan_tree(P.sqrt_filter_combine, sq)
    p2 = P.scan_tree(P.sqrt_filter_combine, [tuple(z)] + sq[1:])
    for a, b in zip(p1, p2):
        np.testing.assert_allclose(a[1], b[1], atol=1e-12)
        np.testing.assert_allclose(a[2] @ a[2].T, b[2] @ b[2].T, atol=1e-12)


def test_smoother_operator_associative():
    rng = np.random.default_rng(15)
    els = [(0.5 * rng.standard_normal((4, 4)), rng.standard_normal(4),
            np.tril(rng.standard_normal((4, 4)))) for _ in range(3)]
    a, b, c = els
    l = P.sqrt_smoother_combine(P.sqrt_smoother_combine(a, b), c)
    r = P.sqrt_smoother_combine(a, P.sqrt_smoother_combine(b, c))
    np.testing.assert_allclose(l[0], r[0], atol=1e-12)
    np.testing.assert_allclose(l[1], r[1], atol=1e-12)
    np.testing.assert_allclose(l[2] @ l[2].T, r[2] @ r[2].T, atol=1e-12)


def test_offsets_change_only_the_mean_parts():
    """The principle the refinement passes' mean-only scans rest on: with F,
    S_Q, H, S_R and N_0 fixed, the offsets c, d, the data y and the prior
    mean enter the filtering elements (Lemma 1, Tables 1-2) and the
    smoothing elements (Lemma 3, Table 4) only through b, eta resp. g, so a
    second pass on another set of offsets has the same A, U, Z, E, D in
    every element and every combine of every scan order (here exactly:
    the same arithmetic on the same factors), and Table 3's b_ij, eta_ij
    are affine in the operands' (b, eta) with coefficients fixed by the
    factors."""
    m = _model(12, 5, 2, seed=21)
    rng = np.random.default_rng(22)
    m2 = dict(m)
    m2["c"] = m["c"] + rng.standard_normal(m["c"].shape)
    m2["d"] = m["d"] + rng.standard_normal(m["d"].shape)
    m2["y"] = m["y"] + rng.standard_normal(m["y"].shape)
    m2["m0"] = m["m0"] + rng.standard_normal(m["m0"].shape)
    e1, _ = _elements(m)
    e2, _ = _elements(m2)
    for a, b in zip(e1, e2):
        for k in (0, 2, 4):                      # A, U, Z
            assert np.array_equal(a[k], b[k])
        assert not np.allclose(a[1], b[1])       # b moves
    for scan in (P.scan_sequential, P.scan_tree):
        p1, p2 = scan(P.sqrt_filter_combine, e1), scan(P.sqrt_filter_combine, e2)
        for a, b in zip(p1, p2):
            for k in (0, 2, 4):
                assert np.array_equal(a[k], b[k])
    # b_ij, eta_ij affine in the operands' (b, eta): second differences vanish
    ei, ej = e1[3], e1[4]
    def mean_part(db_i, de_i, db_j, de_j):
        out = P.sqrt_filter_combine((ei[0], ei[1] + db_i, ei[2], ei[3] + de_i, ei[4]),
                                    (ej[0], ej[1] + db_j, ej[2], ej[3] + de_j, ej[4]))
        return np.concatenate([out[1], out[3]])
    u = [rng.standard_normal(5) for _ in range(4)]
    v = [rng.standard_normal(5) for _ in range(4)]
    f0 = mean_part(*[np.zeros(5)] * 4)
    fu, fv = mean_part(*u), mean_part(*v)
    fuv = mean_part(*[a + b for a, b in zip(u, v)])
    np.testing.assert_allclose(fuv - f0, (fu - f0) + (fv - f0), atol=1e-10)
    f2u = mean_part(*[2 * a for a in u])
    np.testing.assert_allclose(f2u - f0, 2 * (fu - f0), atol=1e-10)
    # smoothing elements: E, D fixed by F, S_Q and the filter factor
    Nf = np.tril(rng.standard_normal((5, 5))) + 3 * np.eye(5)
    s1 = P.sqrt_smoother_element(m["F"][2], m["c"][2], m["SQ"][2], rng.standard_normal(5), Nf)
    s2 = P.sqrt_smoother_element(m["F"][2], m2["c"][2], m["SQ"][2], rng.standard_normal(5), Nf)
    assert np.array_equal(s1[0], s2[0]) and np.array_equal(s1[2], s2[2])
    assert not np.allclose(s1[1], s2[1])
