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


def test_std_rejects_extended(B, ctx):
    import ctypes
    d = W.ct_batch(lengths=[10], seed=1)
    f32 = torch.float32
    y, m0, P0 = _dev(d["y"], f32), _dev(d["m0"], f32), _dev(_P0(d), f32)
    ms = torch.empty((11, 5), device="cuda:0")
    Ps = torch.empty((11, 5, 5), device="cuda:0")
    mdl = B._model(d["dt"], np.array([[-1.5, 0.5], [1.0, 1.0]]))
    off = (ctypes.c_int64 * 2)(0, 10)
    th = (ctypes.c_double * 3)(*[float(v) for v in d["theta"]])
    rc = B.lib.sqsm_ipls_smooth_std(ctx.h, B.F32, ctypes.byref(mdl), th, B.EXTENDED, 2, 1, off,
                                    y.data_ptr(), m0.data_ptr(), P0.data_ptr(), ms.data_ptr(),
                                    Ps.data_ptr(), None, None)
    assert rc == B.ERR_UNSUPPORTED
