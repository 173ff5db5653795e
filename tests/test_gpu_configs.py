"""Parity cases at the sizes of the benchmark configurations: coordinated-turn
IPLS at n = 1e4 (M = 10), the length sweep n = 2^10 .. 2^20 (cubature and
extended, FP32 and FP64), the full 4096-sequence ragged batch, and the
gradient of the negative pseudo log-likelihood on 256 sequences of 2000 steps
(against central differences, h = 1e-4) with 50 L-BFGS steps from a
perturbed theta.  Where the FP64 oracle cannot run the whole case, it checks
sampled sequences or the linear smoother of the GPU's own linearisation, and
FP32 is checked against the FP64 build."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ipls as O, models as OM
from oracle.kalman import sqrt_filter_smoother
from paper_2207_00426_gb300 import workloads as W
from gpu_util import rel_mean_err, rel_cov_err, TOL

LIN = {"cubature": 0, "extended": 1}


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _smooth(B, ctx, d, dtype, M, method, offsets=None):
    off = [0, len(d["y"])] if offsets is None else offsets
    m0 = d["m0"] if d["m0"].ndim == 2 else d["m0"][None]
    N0 = d["N0"] if d["N0"].ndim == 3 else d["N0"][None]
    ms, Ns, ll = B.sqsm_ipls_smooth(ctx, d["theta"], _dev(d["y"], dtype), off, _dev(m0, dtype),
                                    _dev(N0, dtype), M, LIN[method], dt=d["dt"])
    torch.cuda.synchronize()
    return ms.double().cpu().numpy(), Ns.double().cpu().numpy(), ll.double().cpu().numpy()


def test_ct_n1e4_m10(B, ctx):
    """n = 1e4, M = 10, FP32: the tenth iteration equals the linear smoother
    of the ninth iteration's linearisation, which matches the sequential FP64
    oracle; FP32 against the FP64 build of the whole run."""
    n, M = 10_000, 10
    d = W.ct_sequence(n=n, seed=1)
    f32 = torch.float32
    y, m0, N0 = _dev(d["y"], f32), _dev(d["m0"][None], f32), _dev(d["N0"][None], f32)
    ms9, Ns9, _ = B.sqsm_ipls_smooth(ctx, d["theta"], y, [0, n], m0, N0, M - 1, 0, dt=d["dt"])
    G = B.sqsm_ct_linearize(ctx, d["theta"], y, [0, n], ms9, Ns9, 0, dt=d["dt"])
    _, _, msl, Nsl, lll = B.sqsm_lgssm_smooth(ctx, *G, m0[0], N0[0], y)
    torch.cuda.synchronize()
    Gn = [g.double().cpu().numpy() for g in G]
    ref = sqrt_filter_smoother(*Gn, d["y"], d["m0"], d["N0"])
    assert rel_mean_err(msl.double().cpu().numpy(), ref[2]) < 1e-4
    assert rel_cov_err(Nsl.double().cpu().numpy(), ref[3]) < 1e-4
    assert abs(lll.item() - ref[4]) < 1e-5 * abs(ref[4])
    ms32, _, ll32 = _smooth(B, ctx, d, f32, M, "cubature")
    ms64, _, ll64 = _smooth(B, ctx, d, torch.float64, M, "cubature")
    assert rel_mean_err(ms32, ms64) < 1e-4
    assert abs(ll32[0] - ll64[0]) < 1e-5 * abs(ll64[0])


@pytest.mark.parametrize("method", ["cubature", "extended"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_sweep_n1024_against_oracle(B, ctx, method, prec):
    n, M = 1024, 4
    d = W.ct_sequence(n=n, seed=2 + 10)
    dtype = torch.float32 if prec == "f32" else torch.float64
    ms, Ns, ll = _smooth(B, ctx, d, dtype, M, method)
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    rms, rNs, rll, _ = O.ipls(ct, d["y"], d["m0"], d["N0"], M, method)
    tol = TOL[prec]
    assert rel_mean_err(ms, rms) < tol["mean"]
    assert rel_cov_err(Ns, rNs) < tol["cov"]
    assert abs(ll[0] - rll) <= (1e-9 if prec == "f64" else 1e-5) * abs(rll)


@pytest.mark.parametrize("method", ["cubature", "extended"])
def test_sweep_n2pow20_f32_against_f64(B, ctx, method):
    n, M = 1 << 20, 2
    d = W.ct_sequence(n=n, seed=2 + 20)
    ms32, Ns32, ll32 = _smooth(B, ctx, d, torch.float32, M, method)
    ms64, Ns64, ll64 = _smooth(B, ctx, d, torch.float64, M, method)
    assert np.all(np.isfinite(ms32)) and ctx.status() == 0
    assert rel_mean_err(ms32, ms64) < 1e-4
    assert rel_cov_err(Ns32, Ns64) < 1e-4
    assert abs(ll32[0] - ll64[0]) < 1e-5 * abs(ll64[0])


def test_batch_4096_ragged(B, ctx):
    """4096 sequences, lengths U{100..5000}, M = 10, FP32: the three shortest
    sequences against the oracle's IPLS; for sampled sequences of every
    length, the tenth iteration against the oracle's sequential smoother of
    the GPU's own linearisation at the ninth iteration (a check that does not
    depend on whether Alg. 3 has converged for that sequence)."""
    d = W.ct_batch(batch=4096, lo=100, hi=5000, seed=3)
    off = [int(v) for v in d["offsets"]]
    lengths = np.diff(d["offsets"])
    M = 10
    ms, Ns, ll = _smooth(B, ctx, d, torch.float32, M, "cubature", off)
    assert np.all(np.isfinite(ms)) and np.all(np.isfinite(ll)) and ctx.status() == 0
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    order = np.argsort(lengths)
    for b in order[:3]:
        yb = d["y"][off[b]:off[b + 1]]
        rms, rNs, rll, _ = O.ipls(ct, yb, d["m0"][b], d["N0"][b], M, "cubature")
        rows = slice(off[b] + b, off[b + 1] + b + 1)
        assert rel_mean_err(ms[rows], rms) < TOL["f32"]["mean"]
        assert rel_cov_err(Ns[rows], rNs) < 1e-4
        assert abs(ll[b] - rll) <= 1e-5 * abs(rll)
    f32 = torch.float32
    y = _dev(d["y"], f32)
    ms9, Ns9, _ = B.sqsm_ipls_smooth(ctx, d["theta"], y, off, _dev(d["m0"], f32), _dev(d["N0"], f32),
                                     M - 1, 0, dt=d["dt"])
    G = B.sqsm_ct_linearize(ctx, d["theta"], y, off, ms9, Ns9, 0, dt=d["dt"])
    torch.cuda.synchronize()
    Gn = [g.double().cpu().numpy() for g in G]
    rng = np.random.default_rng(0)
    for b in list(order[-2:]) + list(rng.choice(4096, 3, replace=False)):
        steps = slice(off[b], off[b + 1])
        rows = slice(off[b] + b, off[b + 1] + b + 1)
        ref = sqrt_filter_smoother(*[g[steps] for g in Gn], d["y"][steps], d["m0"][b], d["N0"][b])
        assert rel_mean_err(ms[rows], ref[2]) < 1e-4
        assert rel_cov_err(Ns[rows], ref[3]) < 1e-4
        assert abs(ll[b] - ref[4]) <= 1e-5 * abs(ref[4])


def _nll(B, c, th, y, off, m0, N0, M, dt):
    nll, grad, change, _, _ = B.sqsm_ipls_nll_grad(c, th, y, off, m0, N0, M, M, dt=dt)
    torch.cuda.synchronize()
    return nll.item(), grad.cpu().numpy(), change.item()


def test_gradient_256x2000_against_central_differences(B, ctx):
    """The gradient of Sec. 5.2 is the derivative at the fixed point of
    Alg. 3; sequences of the batch whose M = 30 iterations have not reached
    it (max-norm change of m^s > 1e-9 from iteration 30 to 31, FP64) are left
    out, and at least half of the 256 must remain."""
    full = W.ct_batch(lengths=[2000] * 256, seed=4)
    f64 = torch.float64
    M = 30
    th = np.asarray(full["theta"]) + np.array([0.1, -0.1, 0.1])
    yf, m0f, N0f = _dev(full["y"], f64), _dev(full["m0"], f64), _dev(full["N0"], f64)
    offf = [int(v) for v in full["offsets"]]
    a, _, _ = B.sqsm_ipls_smooth(ctx, th, yf, offf, m0f, N0f, M, 0, dt=full["dt"])
    b, _, _ = B.sqsm_ipls_smooth(ctx, th, yf, offf, m0f, N0f, M + 1, 0, dt=full["dt"])
    torch.cuda.synchronize()
    dm = (a - b).abs().amax(dim=1).cpu().numpy()
    keep = [i for i in range(256) if dm[offf[i] + i:offf[i + 1] + i + 1].max() < 1e-9]
    assert len(keep) >= 128, len(keep)
    y = _dev(np.concatenate([full["y"][offf[i]:offf[i + 1]] for i in keep]), f64)
    m0, N0 = _dev(full["m0"][keep], f64), _dev(full["N0"][keep], f64)
    off = [2000 * i for i in range(len(keep) + 1)]
    d = {"dt": full["dt"]}
    v, g, change = _nll(B, ctx, th, y, off, m0, N0, M, d["dt"])
    assert change < 1e-6
    h = 1e-4
    fd = np.zeros(3)
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd[i] = (_nll(B, ctx, th + e, y, off, m0, N0, M, d["dt"])[0] -
                 _nll(B, ctx, th - e, y, off, m0, N0, M, d["dt"])[0]) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-3 * np.linalg.norm(fd), (g, fd)
    # FP32 gradient against the FP64 one
    f32 = torch.float32
    _, g32, _ = _nll(B, ctx, th, y.float(), off, m0.float(), N0.float(), M, d["dt"])
    assert np.linalg.norm(g32 - g) <= 1e-3 * np.linalg.norm(g)


def test_lbfgs_50_steps(B, ctx):
    """50 L-BFGS iterations (torch.optim.LBFGS on the autograd function) from
    theta* + (0.3, -0.3, 0.3): the objective decreases and the gradient at
    the end is small against the starting one."""
    from paper_2207_00426_gb300.autograd import ipls_nll
    d = W.ct_batch(lengths=[400] * 16, seed=44)
    f64 = torch.float64
    y, m0, N0 = _dev(d["y"], f64), _dev(d["m0"], f64), _dev(d["N0"], f64)
    off = [int(v) for v in d["offsets"]]
    theta = torch.tensor(np.asarray(d["theta"]) + np.array([0.3, -0.3, 0.3]), dtype=f64,
                         requires_grad=True)
    opt = torch.optim.LBFGS([theta], lr=1.0, max_iter=50, line_search_fn="strong_wolfe")
    vals = []

    def closure():
        opt.zero_grad()
        v = ipls_nll(theta, ctx, y, off, m0, N0, M=20, adj_iters=20, dt=d["dt"])
        v.backward()
        vals.append(v.item())
        return v

    g0 = None
    theta0 = theta.detach().clone()
    v0 = closure()
    g0 = theta.grad.detach().clone()
    opt.step(closure)
    closure()
    g1 = theta.grad.detach().clone()
    assert vals[-1] < v0.item()
    assert torch.linalg.norm(g1) < 1e-3 * torch.linalg.norm(g0), (theta0, theta, g0, g1)
