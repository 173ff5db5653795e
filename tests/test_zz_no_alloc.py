"""sqsm_lgssm_smooth_noalloc: the context-free linear smoother whose scratch
is a fixed array inside the library, for callers that may not allocate
device memory (allocator callbacks, pre-reserved or real-time processes).

Checked through the C ABI against sqsm_lgssm_smooth on two calls in a row
(the second with another model, so stale scratch from the first call would
show), and for the size limit.  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_00426_gb300 import workloads as W
from gpu_util import rel_mean_err, rel_cov_err, TOL


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


def _tensors(m, dtype):
    return {k: torch.tensor(np.ascontiguousarray(v), dtype=dtype, device="cuda:0")
            for k, v in m.items() if k != "x"}


def _noalloc(B, t, n, nx):
    dt = t["y"].dtype
    dev = t["y"].device
    mf = torch.empty((n + 1, nx), dtype=dt, device=dev)
    Nf = torch.empty((n + 1, nx, nx), dtype=dt, device=dev)
    ms = torch.empty((n + 1, nx), dtype=dt, device=dev)
    Ns = torch.empty((n + 1, nx, nx), dtype=dt, device=dev)
    ll = torch.empty(1, dtype=torch.float64, device=dev)
    args = []
    for k in ("F", "c", "SQ", "H", "d", "SR"):
        args += [t[k].data_ptr(), t[k][0].numel()]
    rc = B.lib.sqsm_lgssm_smooth_noalloc(
        0 if dt == torch.float32 else 1, nx, t["y"].shape[1], n, *args, t["m0"].data_ptr(),
        t["N0"].data_ptr(), t["y"].data_ptr(), mf.data_ptr(), Nf.data_ptr(), ms.data_ptr(),
        Ns.data_ptr(), ll.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, (mf, Nf, ms, Ns, ll)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_matches_context_path_twice(B, prec):
    dtype = torch.float32 if prec == "f32" else torch.float64
    ctx = B.Context(0)
    for seed, (n, nx, ny) in ((1, (3000, 5, 2)), (2, (777, 4, 2))):
        m = W.random_lgssm(n, nx, ny, seed=seed)
        t = _tensors(m, dtype)
        rc, got = _noalloc(B, t, n, nx)
        assert rc == B.OK
        ref = B.sqsm_lgssm_smooth(ctx, t["F"], t["c"], t["SQ"], t["H"], t["d"], t["SR"],
                                  t["m0"], t["N0"], t["y"])
        torch.cuda.synchronize()
        got = [g.cpu().numpy() for g in got]
        ref = [r.cpu().numpy() for r in ref]
        tol = TOL[prec]
        assert rel_mean_err(got[0], ref[0]) <= tol["mean"]
        assert rel_mean_err(got[2], ref[2]) <= tol["mean"]
        assert rel_cov_err(got[1], ref[1]) <= tol["cov"]
        assert rel_cov_err(got[3], ref[3]) <= tol["cov"]
        assert abs(got[4][0] - ref[4][0]) <= tol["ll"] * abs(ref[4][0])
    ctx.close()


def test_noalloc_rejects_too_large(B):
    n = 10_000_000
    t = {k: torch.zeros(1, device="cuda:0") for k in ("F", "c", "SQ", "H", "d", "SR", "m0", "N0", "y")}
    p = t["y"].data_ptr()
    rc = B.lib.sqsm_lgssm_smooth_noalloc(0, 5, 2, n, *([p, 0] * 6), p, p, p, p, p, p, p, None,
                                         torch.cuda.current_stream().cuda_stream)
    assert rc == B.ERR_TOO_LARGE
