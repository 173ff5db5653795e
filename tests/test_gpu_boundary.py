"""Boundary behaviour of the C ABI on the GPU:

- argument errors found on the host before any GPU work: offsets that do
  not start at 0, a zero-length segment, decreasing offsets, a pointer that
  is not a multiple of its element size;
- the prior_covariance option: N0 arguments read as covariances P0 and
  factored on the GPU in FP64 (N0 = chol(P0)) give the results of the
  factor path; a P0 that is not positive definite sets SQSM_ERR_NOT_PD;
- sqsm_ipls_nll_grad's fixed-point check: SQSM_ERR_NOT_CONVERGED when the
  trajectory or the adjoint has not settled to tol, none when both have;
- the per-kernel event profiler, with and without graphs."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_00426_gb300 import workloads as W
from gpu_util import rel_mean_err, rel_cov_err


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _ipls_raw(B, ctx, offsets, y, m0, N0, ms, Ns, ll, dtype=0):
    mdl, th = B._ct_model(W.CT_THETA_TRUE, 0.01, W.CT_SENSORS)
    off = (ctypes.c_int64 * len(offsets))(*offsets)
    return B.lib.sqsm_ipls_smooth(ctx.h, dtype, ctypes.byref(mdl), th, B.CUBATURE, 2,
                                  len(offsets) - 1, off, y, m0, N0, None, None, ms, Ns, ll,
                                  torch.cuda.current_stream().cuda_stream)


def test_bad_offsets_are_refused_on_the_host(B):
    ctx = B.Context(0)
    buf = torch.zeros(4096, dtype=torch.float32, device="cuda:0")
    p = buf.data_ptr()
    ll = torch.zeros(8, dtype=torch.float64, device="cuda:0").data_ptr()
    for offs in ([1, 10], [0, 10, 10, 20], [0, 10, 5], [0, 0], [-1, 10]):
        assert _ipls_raw(B, ctx, offs, p, p, p, p, p, ll) == B.ERR_INVALID_ARG, offs
        assert "offsets" in B.lib.sqsm_last_error(ctx.h).decode()
    # the same buffers with valid offsets run
    assert _ipls_raw(B, ctx, [0, 10, 20], p, p, p, p, p, ll) == B.OK
    torch.cuda.synchronize()
    ctx.status()
    ctx.close()


def test_misaligned_pointers_are_refused_on_the_host(B):
    ctx = B.Context(0)
    buf = torch.zeros(4096, dtype=torch.float64, device="cuda:0")
    p = buf.data_ptr()
    ll = torch.zeros(8, dtype=torch.float64, device="cuda:0").data_ptr()
    for i in range(5):
        args = [p] * 5
        args[i] = p + 2
        assert _ipls_raw(B, ctx, [0, 10], *args, ll) == B.ERR_INVALID_ARG, i
        assert _ipls_raw(B, ctx, [0, 10], *args, ll, dtype=1) == B.ERR_INVALID_ARG, i
    assert _ipls_raw(B, ctx, [0, 10], p + 4, p, p, p, p, ll, dtype=1) == B.ERR_INVALID_ARG
    assert _ipls_raw(B, ctx, [0, 10], p, p, p, p, p, ll + 4) == B.ERR_INVALID_ARG
    assert "element size" in B.lib.sqsm_last_error(ctx.h).decode()
    # linear smoother: misaligned observation array
    m = W.random_lgssm(20, 4, 2, seed=3)
    t = {k: _dev(v, torch.float32) for k, v in m.items() if k != "x"}
    yb = torch.zeros(41, dtype=torch.float32, device="cuda:0")
    ymis = yb[1:].view(20, 2)       # 4-byte aligned: fine for FP32
    B.sqsm_lgssm_smooth(ctx, t["F"], t["c"], t["SQ"], t["H"], t["d"], t["SR"], t["m0"], t["N0"],
                        ymis)
    torch.cuda.synchronize()
    raw = yb.data_ptr() + 2
    outs = [torch.empty(s, dtype=torch.float32, device="cuda:0").data_ptr()
            for s in ((21, 4), (21, 4, 4), (21, 4), (21, 4, 4))]
    args = []
    for k in ("F", "c", "SQ", "H", "d", "SR"):
        args += [t[k].data_ptr(), t[k][0].numel()]
    rc = B.lib.sqsm_lgssm_smooth(ctx.h, 0, 4, 2, 20, *args, t["m0"].data_ptr(),
                                 t["N0"].data_ptr(), raw, *outs, None,
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == B.ERR_INVALID_ARG
    ctx.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_prior_covariance_matches_factor(B, prec):
    dtype = torch.float32 if prec == "f32" else torch.float64
    tol = 1e-5 if prec == "f32" else 1e-12
    d = W.ct_batch(lengths=[300, 57, 1000], seed=21)
    y, m0, N0 = (_dev(d[k], dtype) for k in ("y", "m0", "N0"))
    # a full prior covariance per sequence (the workload's N0 is diagonal)
    rng = np.random.default_rng(5)
    N0full = np.stack([np.tril(0.02 * rng.standard_normal((5, 5))) + 0.1 * np.eye(5)
                       for _ in range(3)])
    P0 = N0full @ np.swapaxes(N0full, 1, 2)
    N0f, P0d = _dev(N0full, dtype), _dev(P0, dtype)
    cf = B.Context(0)
    cp = B.Context(0, prior_covariance=True)
    a = B.sqsm_ipls_smooth(cf, d["theta"], y, d["offsets"], m0, N0f, 4, dt=d["dt"])
    b = B.sqsm_ipls_smooth(cp, d["theta"], y, d["offsets"], m0, P0d, 4, dt=d["dt"])
    torch.cuda.synchronize()
    assert rel_mean_err(b[0].cpu().numpy(), a[0].cpu().numpy()) < tol
    assert rel_cov_err(b[1].cpu().numpy(), a[1].cpu().numpy()) < tol
    assert np.allclose(b[2].cpu().numpy(), a[2].cpu().numpy(), rtol=tol, atol=0)
    # tolerance mode and NLL + gradient take the option too
    at = B.sqsm_ipls_smooth_tol(cf, d["theta"], y, d["offsets"], m0, N0f, 6, 0.0, dt=d["dt"])
    bt = B.sqsm_ipls_smooth_tol(cp, d["theta"], y, d["offsets"], m0, P0d, 6, 0.0, dt=d["dt"])
    ag = B.sqsm_ipls_nll_grad(cf, d["theta"], y, d["offsets"], m0, N0f, 4, 4, dt=d["dt"])
    bg = B.sqsm_ipls_nll_grad(cp, d["theta"], y, d["offsets"], m0, P0d, 4, 4, dt=d["dt"])
    torch.cuda.synchronize()
    assert rel_mean_err(bt[0].cpu().numpy(), at[0].cpu().numpy()) < tol
    assert abs(bg[0].item() - ag[0].item()) <= tol * abs(ag[0].item())
    assert np.allclose(bg[1].cpu().numpy(), ag[1].cpu().numpy(), rtol=1e3 * tol, atol=0)
    assert cp.status() == 0 and cf.status() == 0
    # linear smoother
    m = W.random_lgssm(200, 4, 2, seed=6)
    t = {k: _dev(v, dtype) for k, v in m.items() if k != "x"}
    P0l = _dev(m["N0"] @ m["N0"].T, dtype)
    ra = B.sqsm_lgssm_smooth(cf, t["F"], t["c"], t["SQ"], t["H"], t["d"], t["SR"], t["m0"],
                             t["N0"], t["y"])
    rb = B.sqsm_lgssm_smooth(cp, t["F"], t["c"], t["SQ"], t["H"], t["d"], t["SR"], t["m0"], P0l,
                             t["y"])
    torch.cuda.synchronize()
    assert rel_mean_err(rb[2].cpu().numpy(), ra[2].cpu().numpy()) < tol
    assert abs(rb[4].item() - ra[4].item()) <= tol * abs(ra[4].item())
    cf.close()
    cp.close()


def test_prior_not_positive_definite_sets_not_pd(B):
    d = W.ct_batch(lengths=[50, 60], seed=22)
    f64 = torch.float64
    y, m0 = _dev(d["y"], f64), _dev(d["m0"], f64)
    P0 = np.stack([0.01 * np.eye(5), 0.01 * np.eye(5)])
    P0[1, 2, 2] = -1e-4                      # second prior indefinite
    cp = B.Context(0, prior_covariance=True)
    ms, Ns, ll = B.sqsm_ipls_smooth(cp, d["theta"], y, d["offsets"], m0, _dev(P0, f64), 2,
                                    dt=d["dt"])
    torch.cuda.synchronize()
    st = cp.status()
    assert st & B.ERR_NOT_PD
    llh = ll.cpu().numpy()
    assert np.isfinite(llh[0]) and not np.isfinite(llh[1])
    # a valid prior afterwards clears nothing by itself but raises nothing new
    P0[1, 2, 2] = 1e-2
    B.sqsm_ipls_smooth(cp, d["theta"], y, d["offsets"], m0, _dev(P0, f64), 2, dt=d["dt"])
    torch.cuda.synchronize()
    assert cp.status() == 0
    cp.close()


def test_nll_grad_fixed_point_check(B):
    f64 = torch.float64
    ctx = B.Context(0)
    # a short sequence that converges: no flag at tol 1e-6 after 40 + 40 iterations
    d = W.ct_batch(lengths=[300], seed=4)
    y, m0, N0 = (_dev(d[k], f64) for k in ("y", "m0", "N0"))
    ich = torch.empty(1, dtype=f64, device="cuda:0")
    nll, g, ch, _, _ = B.sqsm_ipls_nll_grad(ctx, d["theta"], y, d["offsets"], m0, N0, 40, 40,
                                            dt=d["dt"], tol=1e-6, ipls_change=ich)
    torch.cuda.synchronize()
    nll40 = nll.item()
    assert ich.item() < 1e-6 and ch.item() < 1e-6
    assert ctx.status() == 0
    # too few iterations: both changes large, flag set
    nll, g, ch, _, _ = B.sqsm_ipls_nll_grad(ctx, d["theta"], y, d["offsets"], m0, N0, 1, 2,
                                            dt=d["dt"], tol=1e-6, ipls_change=ich)
    torch.cuda.synchronize()
    assert ich.item() > 1e-6 and ch.item() > 1e-6
    assert ctx.status() == B.ERR_NOT_CONVERGED
    # tol <= 0: no check
    B.sqsm_ipls_nll_grad(ctx, d["theta"], y, d["offsets"], m0, N0, 1, 2, dt=d["dt"], tol=0.0)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    # adj_iters = 0: the same NLL as with the adjoint, grad zero, adjoint
    # change reported as 0
    nll0, g0, ch0, _, _ = B.sqsm_ipls_nll_grad(ctx, d["theta"], y, d["offsets"], m0, N0, 40, 0,
                                               dt=d["dt"])
    torch.cuda.synchronize()
    assert abs(nll0.item() - nll40) <= 1e-12 * abs(nll40)
    assert np.all(g0.cpu().numpy() == 0) and ch0.item() == 0.0
    ctx.close()


def test_profiler_times_every_launch(B):
    """sqsm_profile_enable / sqsm_profile_read with and without graphs: the
    same kernel families and launch counts in both modes, each family's
    time positive, and their sum within the call's own event time."""
    d = W.ct_batch(lengths=[3000, 1700], seed=8)
    f32 = torch.float32
    y, m0, N0 = (_dev(d[k], f32) for k in ("y", "m0", "N0"))
    counts = {}
    for graph in (False, True):
        ctx = B.Context(0, use_graph=graph)
        call = lambda: B.sqsm_ipls_smooth(ctx, d["theta"], y, d["offsets"], m0, N0, 3, dt=d["dt"])
        call()
        torch.cuda.synchronize()
        ctx.profile(True)
        call()    # builds the instrumented graph (graph mode)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        call()
        b.record()
        torch.cuda.synchronize()
        fam = ctx.profile_read()
        ctx.profile(False)
        assert ctx.status() == 0
        ctx.close()
        assert {"ct_slr", "filter_leaf_up", "filter_leaf_down", "smoother_leaf_up",
                "smoother_leaf_down", "loglik_reduce"} <= set(fam), fam
        assert all(t > 0 and c > 0 for t, c in fam.values())
        assert fam["ct_slr"][1] == 3 and fam["filter_leaf_up"][1] == 3   # one per iteration
        assert sum(t for t, _ in fam.values()) <= 1.05 * a.elapsed_time(b) + 0.05
        counts[graph] = {k: c for k, (_, c) in fam.items()}
    assert counts[False] == counts[True]
