"""Alg. 3 run until convergence (sqsm_ipls_smooth_tol): the number of
iterations and the result match the oracle's tolerance mode, the graph
(conditional WHILE node) and host-loop forms agree, and tol = 0 runs exactly
max_iters iterations of the fixed-M smoother."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ipls as O, models as OM
from paper_2207_00426_gb300 import workloads as W
from gpu_util import rel_mean_err, rel_cov_err


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _inputs(d, dtype):
    return _dev(d["y"], dtype), _dev(d["m0"], dtype), _dev(d["N0"], dtype)


@pytest.mark.parametrize("use_graph", [True, False])
def test_iterations_match_oracle(B, use_graph):
    d = W.ct_batch(lengths=[300], seed=4)
    f64 = torch.float64
    c = B.Context(0, use_graph=use_graph)
    y, m0, N0 = _inputs(d, f64)
    tol = 1e-8
    ms, Ns, ll, it = B.sqsm_ipls_smooth_tol(c, d["theta"], y, d["offsets"], m0, N0, 50, tol,
                                            dt=d["dt"])
    torch.cuda.synchronize()
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    rms, rNs, rll, rit = O.ipls(ct, d["y"], d["m0"][0], d["N0"][0], 50, "cubature", tol=tol)
    assert it.item() == rit
    assert 3 < rit < 50
    assert rel_mean_err(ms.cpu().numpy(), rms) < 1e-9
    assert rel_cov_err(Ns.cpu().numpy(), rNs) < 1e-9
    assert abs(ll.item() - rll) <= 1e-9 * abs(rll)
    c.close()


def test_graph_and_host_loop_agree_on_a_batch(B):
    d = W.ct_batch(lengths=[120, 37, 250, 5], seed=8)
    f32 = torch.float32
    y, m0, N0 = _inputs(d, f32)
    out = []
    for use_graph in (True, False):
        c = B.Context(0, use_graph=use_graph)
        r = B.sqsm_ipls_smooth_tol(c, d["theta"], y, d["offsets"], m0, N0, 40, 1e-4, dt=d["dt"])
        torch.cuda.synchronize()
        out.append([t.cpu() for t in r])
        c.close()
    (ms_g, Ns_g, ll_g, it_g), (ms_h, Ns_h, ll_h, it_h) = out
    assert it_g.item() == it_h.item() and 1 < it_g.item() <= 40
    assert torch.equal(ms_g, ms_h) and torch.equal(ll_g, ll_h)


def test_tol_zero_runs_max_iters(B):
    d = W.ct_batch(lengths=[64, 200], seed=9)
    f32 = torch.float32
    y, m0, N0 = _inputs(d, f32)
    c = B.Context(0)
    ms, Ns, ll, it = B.sqsm_ipls_smooth_tol(c, d["theta"], y, d["offsets"], m0, N0, 7, 0.0,
                                            dt=d["dt"])
    ms7, Ns7, ll7 = B.sqsm_ipls_smooth(c, d["theta"], y, d["offsets"], m0, N0, 7, 0, dt=d["dt"])
    torch.cuda.synchronize()
    assert it.item() == 7
    assert torch.equal(ms, ms7) and torch.equal(Ns, Ns7) and torch.equal(ll, ll7)
    # repeated calls replay the cached graph and reset the counters
    _, _, _, it2 = B.sqsm_ipls_smooth_tol(c, d["theta"], y, d["offsets"], m0, N0, 7, 0.0,
                                          dt=d["dt"])
    torch.cuda.synchronize()
    assert it2.item() == 7
    c.close()


def test_invalid_tolerance_arguments(B):
    d = W.ct_batch(lengths=[10], seed=1)
    y, m0, N0 = _inputs(d, torch.float32)
    c = B.Context(0)
    for max_iters, tol in ((0, 1e-3), (5, -1.0), (5, float("nan"))):
        with pytest.raises(B.SqsmError) as e:
            B.sqsm_ipls_smooth_tol(c, d["theta"], y, d["offsets"], m0, N0, max_iters, tol,
                                   dt=d["dt"])
        assert e.value.code == B.ERR_INVALID_ARG
    c.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_refined_tolerance_mode_equals_fixed_m(B, use_graph):
    """FP32 with one refinement pass per iteration (whose filter scan
    replays its top levels mean-only, from shared-memory staged factors; in
    the graph form inside the conditional WHILE node): the tolerance run
    stops where the fixed-M smoother with the same M gives the same means,
    factors and log-likelihood bit for bit.  The 6000-step sequence has a
    three-role chunk level and a top of 63 items (the largest staging)."""
    d = W.ct_batch(lengths=[6000, 300, 45], seed=12)
    f32 = torch.float32
    y, m0, N0 = _inputs(d, f32)
    c = B.Context(0, use_graph=use_graph, refine=1)
    ms, Ns, ll, it = B.sqsm_ipls_smooth_tol(c, d["theta"], y, d["offsets"], m0, N0, 30, 1e-3,
                                            dt=d["dt"])
    torch.cuda.synchronize()
    M = it.item()
    assert 1 < M <= 30 and c.status() == 0
    msM, NsM, llM = B.sqsm_ipls_smooth(c, d["theta"], y, d["offsets"], m0, N0, M, 0, dt=d["dt"])
    torch.cuda.synchronize()
    assert torch.equal(ms, msM) and torch.equal(Ns, NsM) and torch.equal(ll, llM)
    assert torch.isfinite(ms).all()
    c.close()
