"""Parity of the parallel square-root filter + smoother (Alg. 1, Alg. 2) and
log-likelihood against the sequential FP64 oracle, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.kalman import sqrt_filter_smoother
from paper_2207_00426_gb300 import workloads as W
from gpu_util import rel_mean_err, rel_cov_err, TOL


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _run(B, ctx, m, dtype, strides=None):
    dev = torch.device("cuda:0")
    t = {k: torch.tensor(np.ascontiguousarray(v), dtype=dtype, device=dev)
         for k, v in m.items() if k != "x"}
    out = B.sqsm_lgssm_smooth(ctx, t["F"], t["c"], t["SQ"], t["H"], t["d"], t["SR"], t["m0"],
                              t["N0"], t["y"], strides=strides)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out]


def _check(got, m, tol):
    mf, Nf, ms, Ns, ll = got
    ref = sqrt_filter_smoother(m["F"], m["c"], m["SQ"], m["H"], m["d"], m["SR"], m["y"],
                               m["m0"], m["N0"])
    assert rel_mean_err(mf, ref[0]) < tol["mean"]
    assert rel_cov_err(Nf, ref[1]) < tol["cov"]
    assert rel_mean_err(ms, ref[2]) < tol["mean"]
    assert rel_cov_err(Ns, ref[3]) < tol["cov"]
    assert abs(ll[0] - ref[4]) <= tol["ll"] * abs(ref[4])
    assert np.allclose(np.triu(Ns, 1), 0) and np.all(np.diagonal(Ns, axis1=1, axis2=2) >= 0)


SHAPES = [(1, 1), (1, 2), (2, 2), (3, 2), (2, 3), (4, 2), (5, 2), (6, 3)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("n", [1, 2, 5, 17, 130])
def test_random_models(B, ctx, prec, nx, ny, n):
    m = W.random_lgssm(n, nx, ny, seed=n * 31 + nx * 7 + ny)
    got = _run(B, ctx, m, torch.float64 if prec == "f64" else torch.float32)
    _check(got, m, TOL[prec])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_linear_cv_config(B, ctx, prec):
    """n_x = 4, n_y = 2 constant-velocity model, n = 1000."""
    m = W.linear_cv(n=1000, seed=0)
    got = _run(B, ctx, m, torch.float64 if prec == "f64" else torch.float32)
    _check(got, m, TOL[prec])


def test_time_invariant_strides(B, ctx):
    m = W.linear_cv(n=333, seed=4)
    full = _run(B, ctx, m, torch.float64)
    mi = dict(m)
    for k in ("F", "c", "SQ", "H", "d", "SR"):
        mi[k] = m[k][0]
    ti = _run(B, ctx, mi, torch.float64, strides=(0, 0, 0, 0, 0, 0))
    for a, b in zip(full, ti):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("leaf,radix", [(1, 2), (3, 5), (16, 8)])
def test_scan_shapes_agree(B, leaf, radix):
    """Different leaf chunk / radix (different bracketings of the scan)."""
    c2 = B.Context(0, leaf_chunk=leaf, radix=radix)
    m = W.random_lgssm(301, 5, 2, seed=9)
    got = _run(B, c2, m, torch.float64)
    _check(got, m, TOL["f64"])


def test_full_size_random_model_f32(B, ctx):
    """n = 100000 steps, FP32, against the sequential oracle."""
    m = W.random_lgssm(100_000, 5, 2, seed=77)
    got = _run(B, ctx, m, torch.float32)
    _check(got, m, dict(mean=1e-4, cov=1e-4, ll=1e-5))


def test_invalid_arguments(B, ctx):
    dev = torch.device("cuda:0")
    z = torch.zeros((4, 4), device=dev)
    rc = B.lib.sqsm_lgssm_smooth(ctx.h, 0, 4, 2, 0, *([z.data_ptr(), 0] * 6), z.data_ptr(),
                                 z.data_ptr(), z.data_ptr(), None, None, z.data_ptr(),
                                 z.data_ptr(), None, None)
    assert rc == B.ERR_INVALID_ARG
    rc = B.lib.sqsm_lgssm_smooth(ctx.h, 0, 7, 7, 3, *([z.data_ptr(), 0] * 6), z.data_ptr(),
                                 z.data_ptr(), z.data_ptr(), None, None, z.data_ptr(),
                                 z.data_ptr(), None, None)
    assert rc == B.ERR_UNSUPPORTED
    assert "compiled" in B.lib.sqsm_last_error(ctx.h).decode()


@pytest.mark.parametrize("prec,rank,n", [("f64", 0, 30), ("f64", 1, 30), ("f32", 1, 30),
                                         ("f32", 0, 16)])
def test_singular_process_noise(B, ctx, prec, rank, n):
    """A noise factor S_Q of rank 1 or 0 (Q not positive definite): the
    square-root form needs no positive-definite Q (Tria of a rank-deficient
    block, reading 2), and the results equal the oracle's as long as the
    predicted covariances stay positive definite -- here F is invertible and
    P0 positive definite.  With no process noise at all the filter
    covariance collapses as observations accumulate and the FP32 RTS
    smoother loses accuracy with n (sequential or parallel alike: 2e-4 at
    n = 30, diverging by n = 60), so that FP32 case is checked at n = 16."""
    m = W.random_lgssm(n, 4, 2, seed=77 + rank)
    SQ = m["SQ"].copy()
    SQ[:, :, rank:] = 0.0
    # observations of this model (rank-deficient process noise)
    rng = np.random.default_rng(5 + rank)
    x = m["m0"] + m["N0"] @ rng.standard_normal(4)
    y = np.zeros_like(m["y"])
    for t in range(n):
        x = m["F"][t] @ x + m["c"][t] + SQ[t] @ rng.standard_normal(4)
        y[t] = m["H"][t] @ x + m["d"][t] + m["SR"][t] @ rng.standard_normal(2)
    m = dict(m, SQ=SQ, y=y)
    got = _run(B, ctx, m, torch.float64 if prec == "f64" else torch.float32)
    _check(got, m, TOL[prec])


def test_nonfinite_input_sets_status(B):
    c2 = B.Context(0)
    m = W.linear_cv(n=50, seed=1)
    m["y"] = m["y"].copy()
    m["y"][20, 0] = np.nan
    _run(B, c2, m, torch.float32)
    assert c2.status() & B.ERR_NONFINITE
    assert c2.status() == 0
