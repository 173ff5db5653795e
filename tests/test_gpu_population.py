"""Alg. 3 on the Ricker population model with Poisson counts (state-
dependent observation noise, known initial state) against the oracle, in
FP64 and FP32, Taylor and cubature, single and ragged batch, fixed M and
until convergence."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ipls as O, models as OM
from paper_2207_00426_gb300 import workloads as W
from gpu_util import rel_mean_err, rel_cov_err

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


@pytest.mark.parametrize("method", ["cubature", "extended"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_population_matches_oracle(B, ctx, method, prec):
    lengths = [120, 1, 37, 64]
    d = W.ricker_batch(lengths, seed=71)
    dt = torch.float64 if prec == "f64" else torch.float32
    M = 8
    ms, Ns, ll = B.sqsm_ipls_smooth_population(ctx, d["theta"], _dev(d["y"], dt), d["offsets"],
                                               _dev(d["m0"], dt), _dev(d["N0"], dt), M,
                                               LIN[method])
    torch.cuda.synchronize()
    ms, Ns, ll = ms.double().cpu().numpy(), Ns.double().cpu().numpy(), ll.cpu().numpy()
    mdl = OM.RickerPoisson(d["theta"])
    off = d["offsets"]
    tol = 1e-9 if prec == "f64" else 2e-5
    for b in range(len(lengths)):
        yb = d["y"][off[b]:off[b + 1]]
        rms, rNs, rll, _ = O.ipls(mdl, yb, d["m0"][b], d["N0"][b], M, method)
        rows = slice(off[b] + b, off[b + 1] + b + 1)
        assert rel_mean_err(ms[rows], rms) < tol
        assert rel_cov_err(Ns[rows], rNs) < (1e-9 if prec == "f64" else 1e-4)
        assert abs(ll[b] - rll) <= (1e-10 if prec == "f64" else 1e-5) * abs(rll)
    assert ctx.status() == 0


def test_population_until_convergence(B, ctx):
    d = W.ricker_batch([200], seed=72)
    f64 = torch.float64
    ms, Ns, ll, it = B.sqsm_ipls_smooth_population(ctx, d["theta"], _dev(d["y"], f64),
                                                   d["offsets"], _dev(d["m0"], f64),
                                                   _dev(d["N0"], f64), 100, 0, tol=1e-9)
    torch.cuda.synchronize()
    mdl = OM.RickerPoisson(d["theta"])
    rms, _, rll, rit = O.ipls(mdl, d["y"], d["m0"][0], d["N0"][0], 100, "cubature", tol=1e-9)
    assert it.item() == rit < 100
    assert rel_mean_err(ms.cpu().numpy(), rms) < 1e-9
    assert abs(ll.item() - rll) <= 1e-9 * abs(rll)


def test_population_rejected_where_unsupported(B, ctx):
    import ctypes
    d = W.ricker_batch([10], seed=1)
    y = _dev(d["y"], torch.float32)
    m0, N0 = _dev(d["m0"], torch.float32), _dev(d["N0"], torch.float32)
    ms = torch.empty((11, 1), device="cuda:0")
    Ns = torch.empty((11, 1, 1), device="cuda:0")
    mdl = B.Model(B.MODEL_POPULATION, 1.0, (ctypes.c_double * 4)())
    th = (ctypes.c_double * 3)(*[float(v) for v in d["theta"]])
    off = (ctypes.c_int64 * 2)(0, 10)
    # Gauss-Hermite is not offered for this model
    rc = B.lib.sqsm_ipls_smooth(ctx.h, B.F32, ctypes.byref(mdl), th, B.GAUSS_HERMITE, 3, 1, off,
                                y.data_ptr(), m0.data_ptr(), N0.data_ptr(), None, None,
                                ms.data_ptr(), Ns.data_ptr(), None, None)
    assert rc == B.ERR_UNSUPPORTED
    # the CT-only entry points
    rc = B.lib.sqsm_ct_linearize(ctx.h, B.F32, ctypes.byref(mdl), th, 0, 1, off, y.data_ptr(),
                                 ms.data_ptr(), Ns.data_ptr(), *([ms.data_ptr()] * 6), None)
    assert rc == B.ERR_UNSUPPORTED
