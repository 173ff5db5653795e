"""Parity at the benchmark's full size (n = 1e5 coordinated-turn sequence,
seed 1) against stored FP64 oracle values (tests/golden/, written by
tests/golden/make_golden.py from oracle/ only).

- The gradient of the negative pseudo log-likelihood at a frozen trajectory
  (Sec. 5.2 without the fixed-point term: M = 0, one adjoint iteration, so
  lambda = 0): every adjoint map scan and leaf kernel runs at the bench's
  size and scan shape, compared with central differences of the oracle's
  sequential square-root filter on its cubature linearisation."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_00426_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


def _checksum(a):
    a = np.asarray(a, dtype=np.float64)
    return float(np.sum(a * np.arange(1, a.size + 1).reshape(a.shape) / a.size))


@pytest.mark.parametrize("prec,gtol,ltol", [("f64", 1e-6, 1e-10), ("f32", 1e-3, 1e-5)])
def test_frozen_trajectory_gradient_n1e5(B, prec, gtol, ltol):
    g = json.load(open(os.path.join(GOLDEN, "frozen_grad_ct_n1e5_seed1.json")))
    n = 100_000
    d = W.ct_sequence(n=n, seed=1)
    assert np.isclose(_checksum(d["x"]), g["x_checksum"], rtol=1e-12, atol=0)
    assert np.isclose(_checksum(d["y"]), g["y_checksum"], rtol=1e-12, atol=0)
    dt = torch.float32 if prec == "f32" else torch.float64
    dev = "cuda:0"
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    ims = t(d["x"])
    iNs = t(np.tile(0.05 * np.eye(5), (n + 1, 1, 1)))
    ctx = B.Context(0)
    ich = torch.empty(1, dtype=torch.float64, device=dev)
    nll, grad, ch, _, _ = B.sqsm_ipls_nll_grad(ctx, g["theta"], t(d["y"]), [0, n],
                                               t(d["m0"][None]), t(d["N0"][None]), 0, 1,
                                               dt=d["dt"], init_ms=ims, init_Ns=iNs,
                                               ipls_change=ich)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ref = np.array(g["grad_nll"])
    got = grad.cpu().numpy()
    assert np.linalg.norm(got - ref) <= gtol * np.linalg.norm(ref), (got, ref)
    assert abs(nll.item() - g["nll"]) <= ltol * abs(g["nll"]), (nll.item(), g["nll"])
    assert np.isfinite(ich.item())
    ctx.close()


@pytest.mark.parametrize("prec,refine", [("f64", 0), ("f32", 1)])
def test_headline_config_against_oracle(B, prec, refine):
    """Alg. 3 at the benchmark's configuration (n = 1e5, M = 10, cubature,
    prior broadcast as the initial trajectory) against the stored FP64
    oracle run, on every 20th smoothed mean and every 200th factor: FP64 at
    1e-9, FP32 in the benchmark's mode (one refinement pass of each
    iteration's linear smoother) at the 1e-4 / 1e-5 targets."""
    from gpu_util import rel_mean_err, rel_cov_err
    g = np.load(os.path.join(GOLDEN, "ipls_ct_n1e5_seed1_M10.npz"))
    n = int(g["n"])
    d = W.ct_sequence(n=n, seed=int(g["seed"]))
    assert np.isclose(_checksum(d["y"]), float(g["y_checksum"]), rtol=1e-12, atol=0)
    dt = torch.float32 if prec == "f32" else torch.float64
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda:0")
    ctx = B.Context(0, refine=refine)
    ms, Ns, ll = B.sqsm_ipls_smooth(ctx, d["theta"], t(d["y"]), [0, n], t(d["m0"][None]),
                                    t(d["N0"][None]), int(g["M"]), dt=d["dt"])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ms = ms.cpu().numpy()[g["rows_m"]]
    Ns = Ns.cpu().numpy()[g["rows_N"]]
    # means 1e-4 and log-likelihood 1e-5 are the targets; the factors have
    # none, FP32 is held to 5e-4 (measured 1.7e-4 on this non-converging run)
    tol = {"f64": (1e-9, 1e-9, 1e-10), "f32": (1e-4, 5e-4, 1e-5)}[prec]
    em, ec = rel_mean_err(ms, g["ms"]), rel_cov_err(Ns, g["Ns"])
    el = abs(ll.item() - float(g["loglik"])) / abs(float(g["loglik"]))
    assert em <= tol[0] and ec <= tol[1] and el <= tol[2], (em, ec, el)
    ctx.close()
