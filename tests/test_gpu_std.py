"""The standard (covariance) form of Alg. 3 on the GPU (left columns of
Tables 1-5, covariance cubature SLR): FP64 against the oracle's standard
form, against the square-root form at a larger size, and FP32 against FP64
where the FP32 run stays finite."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ipls as O, models as OM
from paper_2207_00426_gb300 import workloads as W
from gpu_util import rel_mean_err


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _P0(d):
    return d["N0"] @ np.swapaxes(d["N0"], 1, 2)


def _rel_cov(P, Pr):
    return np.abs(P - Pr).max() / np.abs(Pr).max()


@pytest.mark.parametrize("lengths", [[40], [1, 2, 17, 33, 9]])
def test_std_f64_matches_oracle(B, ctx, lengths):
    d = W.ct_batch(lengths=lengths, seed=61)
    f64 = torch.float64
    M = 5
    ms, Ps, ll = B.sqsm_ipls_smooth_std(ctx, d["theta"], _dev(d["y"], f64), d["offsets"],
                                        _dev(d["m0"], f64), _dev(_P0(d), f64), M, dt=d["dt"])
    torch.cuda.synchronize()
    ms, Ps, ll = ms.cpu().numpy(), Ps.cpu().numpy(), ll.cpu().numpy()
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    off = d["offsets"]
    for b in range(len(lengths)):
        yb = d["y"][off[b]:off[b + 1]]
        rms, rPs, rll, _ = O.ipls_std(ct, yb, d["m0"][b], _P0(d)[b], M)
        rows = slice(off[b] + b, off[b + 1] + b + 1)
        assert rel_mean_err(ms[rows], rms) < 1e-9
        assert _rel_cov(Ps[rows], rPs) < 1e-9
        assert abs(ll[b] - rll) <= 1e-9 * abs(rll)


def test_std_f64_matches_square_root_form(B, ctx):
    d = W.ct_batch(lengths=[2000, 700], seed=62)
    f64 = torch.float64
    y, m0 = _dev(d["y"], f64), _dev(d["m0"], f64)
    M = 6
    ms, Ps, ll = B.sqsm_ipls_smooth_std(ctx, d["theta"], y, d["offsets"], m0, _dev(_P0(d), f64), M,
                                        dt=d["dt"])
    ms2, Ns2, ll2 = B.sqsm_ipls_smooth(ctx, d["theta"], y, d["offsets"], m0, _dev(d["N0"], f64),
                                       M, 0, dt=d["dt"])
    torch.cuda.synchronize()
    P2 = (Ns2 @ Ns2.transpose(1, 2)).cpu().numpy()
    assert rel_mean_err(ms.cpu().numpy(), ms2.cpu().numpy()) < 1e-8
    assert _rel_cov(Ps.cpu().numpy(), P2) < 1e-8
    np.testing.assert_allclose(ll.cpu().numpy(), ll2.cpu().numpy(), rtol=1e-9)


def test_std_f32_short_sequence_matches_f64(B, ctx):
    d = W.ct_batch(lengths=[100], seed=63)
    M = 5
    out = {}
    for dtp in (torch.float32, torch.float64):
        ms, Ps, ll = B.sqsm_ipls_smooth_std(ctx, d["theta"], _dev(d["y"], dtp), d["offsets"],
                                            _dev(d["m0"], dtp), _dev(_P0(d), dtp), M, dt=d["dt"])
        torch.cuda.synchronize()
        out[dtp] = (ms.double().cpu().numpy(), ll.cpu().numpy())
    (m32, l32), (m64, l64) = out[torch.float32], out[torch.float64]
    assert np.all(np.isfinite(m32))
    assert rel_mean_err(m32, m64) < 1e-3
    assert abs(l32[0] - l64[0]) <= 1e-4 * abs(l64[0])


@pytest.mark.parametrize("method", ["cubature", "extended"])
def test_absolute_coordinates(B, method):
    """The printed absolute form (context option) is the same smoother:
    FP64 square-root and standard forms against the oracle (which smooths in
    absolute coordinates), and the square-root form against its deviation
    form."""
    lin = {"cubature": 0, "extended": 1}[method]
    d = W.ct_batch(lengths=[50, 23], seed=64)
    f64 = torch.float64
    y, m0 = _dev(d["y"], f64), _dev(d["m0"], f64)
    M = 5
    cabs = B.Context(0, absolute=True)
    cdev = B.Context(0)
    ms_a, Ns_a, ll_a = B.sqsm_ipls_smooth(cabs, d["theta"], y, d["offsets"], m0,
                                          _dev(d["N0"], f64), M, lin, dt=d["dt"])
    ms_d, _, ll_d = B.sqsm_ipls_smooth(cdev, d["theta"], y, d["offsets"], m0, _dev(d["N0"], f64),
                                       M, lin, dt=d["dt"])
    ms_s, Ps_s, ll_s = B.sqsm_ipls_smooth_std(cabs, d["theta"], y, d["offsets"], m0,
                                              _dev(_P0(d), f64), M, lin, dt=d["dt"])
    torch.cuda.synchronize()
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    off = d["offsets"]
    for b in range(2):
        yb = d["y"][off[b]:off[b + 1]]
        rms, rNs, rll, _ = O.ipls(ct, yb, d["m0"][b], d["N0"][b], M, method)
        rows = slice(off[b] + b, off[b + 1] + b + 1)
        for ms in (ms_a, ms_d, ms_s):
            assert rel_mean_err(ms[rows].cpu().numpy(), rms) < 1e-9
        assert _rel_cov(Ps_s[rows].cpu().numpy(), rNs @ np.swapaxes(rNs, 1, 2)) < 1e-9
        for ll in (ll_a, ll_d, ll_s):
            assert abs(ll[b].item() - rll) <= 1e-9 * abs(rll)
    cabs.close()
    cdev.close()


def test_textbook_slr_is_the_same_regression(B):
    """The textbook option (sigma-point deviations formed from absolute
    function values, the printed formulas) computes the same cubature
    regression: in FP64 both forms of both smoothers equal the oracle; in
    FP32 on a short sequence it stays finite and near the FP64 run (its
    larger error is what the robustness experiment measures)."""
    d = W.ct_batch(lengths=[50, 23], seed=64)
    f64, f32 = torch.float64, torch.float32
    M = 5
    ctb = B.Context(0, absolute=True, textbook_slr=True)
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    off = d["offsets"]
    ms_q, _, ll_q = B.sqsm_ipls_smooth(ctb, d["theta"], _dev(d["y"], f64), off, _dev(d["m0"], f64),
                                       _dev(d["N0"], f64), M, 0, dt=d["dt"])
    ms_s, _, ll_s = B.sqsm_ipls_smooth_std(ctb, d["theta"], _dev(d["y"], f64), off,
                                           _dev(d["m0"], f64), _dev(_P0(d), f64), M, 0, dt=d["dt"])
    ms32, _, ll32 = B.sqsm_ipls_smooth(ctb, d["theta"], _dev(d["y"], f32), off, _dev(d["m0"], f32),
                                       _dev(d["N0"], f32), M, 0, dt=d["dt"])
    torch.cuda.synchronize()
    for b in range(2):
        yb = d["y"][off[b]:off[b + 1]]
        rms, _, rll, _ = O.ipls(ct, yb, d["m0"][b], d["N0"][b], M, "cubature")
        rows = slice(off[b] + b, off[b + 1] + b + 1)
        for ms in (ms_q, ms_s):
            assert rel_mean_err(ms[rows].cpu().numpy(), rms) < 1e-9
        for ll in (ll_q, ll_s):
            assert abs(ll[b].item() - rll) <= 1e-9 * abs(rll)
        assert rel_mean_err(ms32[rows].double().cpu().numpy(), rms) < 1e-3
    assert ctb.status() == 0
    ctb.close()
