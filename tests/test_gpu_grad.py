"""Gradient of the negative pseudo log-likelihood through the IPLS fixed
point (Sec. 5.2), hand-written adjoint on the GPU, against the oracle's
central finite differences of the converged pseudo log-likelihood."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ipls as O, models as OM
from paper_2207_00426_gb300 import workloads as W

THETA = np.log([0.05, 0.01, 0.1])


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _oracle(d, theta, y=None, m0=None, N0=None):
    y = d["y"] if y is None else y
    m0 = d["m0"] if m0 is None else m0
    N0 = d["N0"] if N0 is None else N0
    nll = O.nll(OM.CTBearings, theta, y, m0, N0, "cubature", tol=1e-13, dt=d["dt"])
    g = O.nll_grad_fd(OM.CTBearings, theta, y, m0, N0, "cubature", h=1e-5, tol=1e-13, dt=d["dt"])
    return nll, g


@pytest.mark.parametrize("prec,tol", [("f64", 1e-6), ("f32", 1e-3)])
@pytest.mark.parametrize("n", [30, 131])
def test_gradient_matches_oracle_fd(B, ctx, prec, tol, n):
    d = W.ct_sequence(n=n, seed=31 + n)
    dt = torch.float64 if prec == "f64" else torch.float32
    theta = THETA + np.array([0.2, -0.3, 0.25])
    nll, grad, change, ms, _ = B.sqsm_ipls_nll_grad(ctx, theta, _dev(d["y"], dt), [0, n],
                                                    _dev(d["m0"][None], dt), _dev(d["N0"][None], dt),
                                                    M=40, adj_iters=40, dt=d["dt"])
    torch.cuda.synchronize()
    rnll, rg = _oracle(d, theta)
    g = grad.cpu().numpy()
    assert abs(nll.item() - rnll) <= (1e-9 if prec == "f64" else 1e-5) * abs(rnll)
    assert np.linalg.norm(g - rg) <= tol * np.linalg.norm(rg), (g, rg)
    assert change.item() < (1e-8 if prec == "f64" else 1e-3)


@pytest.mark.parametrize("leaf,radix", [(4, 4), (2, 3), (12, 4), (200, 4)])
def test_gradient_fold_levels(B, leaf, radix):
    """The adjoint's map scans with every upper level folded (explicit radix)
    instead of warp-scanned; leaf chunks of 12 take the one-thread-per-chunk
    leaf down-sweeps, and 200 > n puts the whole sequence in one chunk (no
    upper levels: the sequential smoother's shape)."""
    c2 = B.Context(0, leaf_chunk=leaf, radix=radix)
    n = 131
    d = W.ct_sequence(n=n, seed=31 + n)
    theta = THETA + np.array([0.2, -0.3, 0.25])
    nll, grad, _, _, _ = B.sqsm_ipls_nll_grad(c2, theta, _dev(d["y"], torch.float64), [0, n],
                                              _dev(d["m0"][None], torch.float64),
                                              _dev(d["N0"][None], torch.float64),
                                              M=40, adj_iters=40, dt=d["dt"])
    torch.cuda.synchronize()
    rnll, rg = _oracle(d, theta)
    assert abs(nll.item() - rnll) <= 1e-9 * abs(rnll)
    assert np.linalg.norm(grad.cpu().numpy() - rg) <= 1e-6 * np.linalg.norm(rg)


def test_batched_gradient_is_sum(B, ctx):
    lengths = [17, 40, 3]
    d = W.ct_batch(lengths=lengths, seed=41)
    dt = torch.float64
    nll, grad, _, _, _ = B.sqsm_ipls_nll_grad(ctx, THETA, _dev(d["y"], dt), d["offsets"],
                                              _dev(d["m0"], dt), _dev(d["N0"], dt), M=40,
                                              adj_iters=40, dt=d["dt"])
    torch.cuda.synchronize()
    off = d["offsets"]
    tot_nll, tot_g = 0.0, np.zeros(3)
    for b in range(len(lengths)):
        rn, rg = _oracle(d, THETA, d["y"][off[b]:off[b + 1]], d["m0"][b], d["N0"][b])
        tot_nll += rn
        tot_g += rg
    assert abs(nll.item() - tot_nll) <= 1e-9 * abs(tot_nll)
    np.testing.assert_allclose(grad.cpu().numpy(), tot_g, rtol=1e-6, atol=1e-8 * np.abs(tot_g).max())


def test_autograd_function(B, ctx):
    from paper_2207_00426_gb300.autograd import ipls_nll
    d = W.ct_sequence(n=50, seed=43)
    dt = torch.float64
    theta = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
    val = ipls_nll(theta, ctx, _dev(d["y"], dt), [0, 50], _dev(d["m0"][None], dt),
                   _dev(d["N0"][None], dt), M=40, adj_iters=40, dt=d["dt"])
    (3.0 * val).backward()
    _, rg = _oracle(d, THETA)
    np.testing.assert_allclose(theta.grad.numpy(), 3.0 * rg, rtol=1e-6, atol=1e-9)


def test_unknown_linearization_is_rejected(B, ctx):
    d = W.ct_sequence(n=10, seed=44)
    dt = torch.float64
    import ctypes
    mdl, th = B._ct_model(THETA, d["dt"], d["sensors"])
    off, batch = B._offsets([0, 10])
    z = torch.zeros(64, dtype=dt, device="cuda:0")
    p = z.data_ptr()
    rc = B.lib.sqsm_ipls_nll_grad(ctx.h, 1, ctypes.byref(mdl), th, 7, 5, 5, 0.0, batch,
                                  off, p, p, p, None, None, p, p, p, p, None, None, None)
    assert rc == B.ERR_INVALID_ARG


RULES = {"extended": 1, "unscented": 2, "gauss-hermite": 3}


@pytest.mark.parametrize("prec,tol", [("f64", 1e-6), ("f32", 1e-3)])
@pytest.mark.parametrize("method", ["extended", "unscented", "gauss-hermite"])
def test_gradient_other_rules_match_oracle_fd(B, ctx, prec, tol, method):
    """The adjoint of the Taylor linearisation (second derivatives of the CT
    transition and bearings contracted with the Jacobian cotangents) and of
    the unscented and Gauss-Hermite regressions (every sigma point's
    cotangent, two passes over the points) against the oracle's central
    differences of the converged pseudo log-likelihood with the same rule
    (Sec. 5.2 for the linearisations of Secs. 4.2, 4.3; the paper's
    sqrt(R_11) study uses all four)."""
    n = 40
    d = W.ct_sequence(n=n, seed=61)
    dt = torch.float64 if prec == "f64" else torch.float32
    theta = THETA + np.array([0.2, -0.3, 0.25])
    nll, grad, change, _, _ = B.sqsm_ipls_nll_grad(
        ctx, theta, _dev(d["y"], dt), [0, n], _dev(d["m0"][None], dt), _dev(d["N0"][None], dt),
        M=40, adj_iters=40, dt=d["dt"], linearization=RULES[method])
    torch.cuda.synchronize()
    rnll = O.nll(OM.CTBearings, theta, d["y"], d["m0"], d["N0"], method, tol=1e-13, dt=d["dt"])
    rg = O.nll_grad_fd(OM.CTBearings, theta, d["y"], d["m0"], d["N0"], method, h=1e-5, tol=1e-13,
                       dt=d["dt"])
    g = grad.cpu().numpy()
    assert abs(nll.item() - rnll) <= (1e-9 if prec == "f64" else 1e-5) * abs(rnll)
    assert np.linalg.norm(g - rg) <= tol * np.linalg.norm(rg), (g, rg)
    assert change.item() < (1e-8 if prec == "f64" else 1e-3)


def test_gradient_matches_oracle_forward_mode(B, ctx):
    """Cubature gradient (FP64) against the oracle's second route, forward
    mode through the fixed point (oracle/forward.py)."""
    from oracle import forward as OF
    n = 25
    d = W.ct_sequence(n=n, seed=62)
    theta = THETA + np.array([-0.1, 0.2, -0.15])
    f64 = torch.float64
    nll, grad, _, _, _ = B.sqsm_ipls_nll_grad(ctx, theta, _dev(d["y"], f64), [0, n],
                                              _dev(d["m0"][None], f64), _dev(d["N0"][None], f64),
                                              M=60, adj_iters=60, dt=d["dt"])
    torch.cuda.synchronize()
    rnll, rg, _ = OF.nll_grad_forward(OM.CTBearings(theta, dt=d["dt"]), d["y"], d["m0"], d["N0"])
    g = grad.cpu().numpy()
    assert abs(nll.item() - rnll) <= 1e-9 * abs(rnll)
    assert np.linalg.norm(g - rg) <= 1e-8 * np.linalg.norm(rg), (g, rg)


THETA_R = np.r_[np.log(0.03), THETA[1:], np.log(0.08)]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-6), ("f32", 1e-3)])
def test_gradient_per_sensor_noise(B, ctx, prec, tol):
    """The model with one noise level per sensor (theta = (log sqrt(R_11),
    log q_c, log q_w, log sqrt(R_22)), Sec. 6.4): nll and the four-entry
    gradient against the oracle's central differences."""
    n = 131
    d = W.ct_sequence(n=n, seed=37)
    dt = torch.float64 if prec == "f64" else torch.float32
    nll, grad, change, _, _ = B.sqsm_ipls_nll_grad(ctx, THETA_R, _dev(d["y"], dt), [0, n],
                                                   _dev(d["m0"][None], dt),
                                                   _dev(d["N0"][None], dt), M=40, adj_iters=40,
                                                   dt=d["dt"])
    torch.cuda.synchronize()
    rnll, rg = _oracle(d, THETA_R)
    g = grad.cpu().numpy()
    assert g.shape == (4,)
    assert abs(nll.item() - rnll) <= (1e-9 if prec == "f64" else 1e-5) * abs(rnll)
    assert np.linalg.norm(g - rg) <= tol * np.linalg.norm(rg), (g, rg)
    assert change.item() < (1e-8 if prec == "f64" else 1e-3)


@pytest.mark.parametrize("method", ["cubature", "extended"])
def test_smoother_per_sensor_noise(B, ctx, method):
    """sqsm_ipls_smooth with the per-sensor model against the oracle (FP64),
    and the shared-noise model is its case sqrt(R_11) = sqrt(R_22)."""
    d = W.ct_sequence(n=97, seed=13)
    f64 = torch.float64
    lin = {"cubature": 0, "extended": 1}[method]
    args = (_dev(d["y"], f64), [0, 97], _dev(d["m0"][None], f64), _dev(d["N0"][None], f64), 6, lin)
    ms, Ns, ll = B.sqsm_ipls_smooth(ctx, THETA_R, *args, dt=d["dt"])
    torch.cuda.synchronize()
    rms, rNs, rll, _ = O.ipls(OM.CTBearings(THETA_R, dt=d["dt"]), d["y"], d["m0"], d["N0"], 6,
                              method)
    P = Ns.cpu().numpy() @ np.swapaxes(Ns.cpu().numpy(), -1, -2)
    Pr = rNs @ np.swapaxes(rNs, -1, -2)
    assert np.linalg.norm(ms.cpu().numpy() - rms, axis=-1).max() <= 1e-9 * np.linalg.norm(rms, axis=-1).max()
    assert np.abs(P - Pr).max() <= 1e-9 * np.abs(Pr).max()
    assert abs(ll.item() - rll) <= 1e-10 * abs(rll)
    th4 = np.r_[THETA, THETA[0]]
    a3 = B.sqsm_ipls_smooth(ctx, THETA, *args, dt=d["dt"])
    a4 = B.sqsm_ipls_smooth(ctx, th4, *args, dt=d["dt"])
    torch.cuda.synchronize()
    for u, v in zip(a3, a4):
        assert torch.equal(u, v)


def test_graph_cache_keys_every_output(B):
    """A second call that keeps ms, Ns and nll but hands new grad / change
    tensors must write those (the captured graph is keyed on every output
    pointer), and give the same values as the first call."""
    c2 = B.Context(0, use_graph=True)
    n = 60
    d = W.ct_sequence(n=n, seed=47)
    f64 = torch.float64
    y, m0, N0 = _dev(d["y"], f64), _dev(d["m0"][None], f64), _dev(d["N0"][None], f64)
    ms = torch.empty((n + 1, 5), dtype=f64, device="cuda:0")
    Ns = torch.empty((n + 1, 5, 5), dtype=f64, device="cuda:0")
    nll = torch.empty(1, dtype=f64, device="cuda:0")
    outs = []
    for _ in range(2):
        g = torch.full((3,), float("nan"), dtype=f64, device="cuda:0")
        ch = torch.full((1,), float("nan"), dtype=f64, device="cuda:0")
        B.sqsm_ipls_nll_grad(c2, THETA, y, [0, n], m0, N0, 30, 30, dt=d["dt"], ms=ms, Ns=Ns,
                             nll=nll, grad=g, change=ch)
        torch.cuda.synchronize()
        outs.append((g.cpu().numpy(), ch.item()))
    c2.close()
    (g1, c1), (g2, c2v) = outs
    assert np.all(np.isfinite(g1)) and np.all(np.isfinite(g2))
    np.testing.assert_array_equal(g1, g2)
    assert c1 == c2v
