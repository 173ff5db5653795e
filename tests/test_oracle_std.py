"""Pins of the oracle's standard (covariance) form of the SLR and of Alg. 3:
it must reproduce the square-root form's products (pinned elsewhere by brute
force, closed forms and textbook recursions), and on a linear model it is
the covariance Kalman/RTS smoother after one iteration."""
import numpy as np

from oracle import ipls as O, models as OM, slr as OS
from oracle.kalman import cov_filter, cov_smoother
from paper_2207_00426_gb300 import workloads as W


def _random_nominal(n, seed):
    rng = np.random.default_rng(seed)
    d = W.ct_sequence(n=n, seed=seed)
    ms = d["x"] + 0.05 * rng.standard_normal(d["x"].shape)
    Ns = np.stack([np.tril(0.02 * rng.standard_normal((5, 5))) + np.diag(rng.uniform(0.05, 0.2, 5))
                   for _ in range(n + 1)])
    return d, ms, Ns


def test_std_linearisation_matches_square_root_form():
    d, ms, Ns = _random_nominal(12, 21)
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    Ps = Ns @ np.swapaxes(Ns, 1, 2)
    F, c, SQ, H, dd, SR = OS.linearize(ct, ms, Ns, d["y"], "cubature")
    Fs, cs, Q, Hs, ds, R = OS.linearize_std(ct, ms, Ps, d["y"])
    np.testing.assert_allclose(Fs, F, atol=1e-10)
    np.testing.assert_allclose(cs, c, atol=1e-10)
    np.testing.assert_allclose(Q, SQ @ np.swapaxes(SQ, 1, 2), atol=1e-12)
    np.testing.assert_allclose(Hs, H, atol=1e-10)
    np.testing.assert_allclose(ds, dd, atol=1e-10)
    np.testing.assert_allclose(R, SR @ np.swapaxes(SR, 1, 2), atol=1e-12)


def test_std_ipls_matches_square_root_ipls():
    d = W.ct_batch(lengths=[40], seed=5)
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    N0 = d["N0"][0]
    ms, Ns, ll, _ = O.ipls(ct, d["y"], d["m0"][0], N0, 6)
    ms2, Ps2, ll2, _ = O.ipls_std(ct, d["y"], d["m0"][0], N0 @ N0.T, 6)
    np.testing.assert_allclose(ms2, ms, atol=1e-9)
    np.testing.assert_allclose(Ps2, Ns @ np.swapaxes(Ns, 1, 2), atol=1e-9)
    assert abs(ll2 - ll) < 1e-9 * abs(ll)
    # same stopping rule
    _, _, _, it1 = O.ipls(ct, d["y"], d["m0"][0], N0, 40, tol=1e-9)
    _, _, _, it2 = O.ipls_std(ct, d["y"], d["m0"][0], N0 @ N0.T, 40, tol=1e-9)
    assert it1 == it2 < 40


def test_std_ipls_linear_model_is_the_covariance_smoother():
    m = W.linear_cv(n=30, seed=2)

    class Lin:
        nx, ny = 4, 2

        def f(self, x):
            return m["F"][0] @ x + m["c"][0]

        def h(self, x):
            return m["H"][0] @ x + m["d"][0]

        def branch(self, v, ref):
            return v

        def SQ(self):
            return m["SQ"][0]

        def SR(self):
            return m["SR"][0]

    P0 = m["N0"] @ m["N0"].T
    ms, Ps, ll, _ = O.ipls_std(Lin(), m["y"], m["m0"], P0, 1)
    Q = m["SQ"] @ np.swapaxes(m["SQ"], 1, 2)
    R = m["SR"] @ np.swapaxes(m["SR"], 1, 2)
    mf, Pf, _, ell = cov_filter(m["F"], m["c"], Q, m["H"], m["d"], R, m["y"], m["m0"], P0)
    rms, rPs = cov_smoother(m["F"], m["c"], Q, mf, Pf)
    np.testing.assert_allclose(ms, rms, atol=1e-9)
    np.testing.assert_allclose(Ps, rPs, atol=1e-9)
    assert abs(ll - ell.sum()) < 1e-9 * abs(ell.sum())
