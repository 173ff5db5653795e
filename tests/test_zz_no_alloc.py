"""sqsm_lgssm_smooth_noalloc: the context-free linear smoother whose scratch
is a fixed array inside the library, for callers that may not allocate
device memory (allocator callbacks, processes whose device memory a
framework reserved up front, real-time loops that cannot take an
allocation's synchronisation).

Checked through the C ABI, on calls in a row whose sizes and models change
(so stale scratch from an earlier call would show):
- bit for bit against sqsm_lgssm_smooth on a context with the same scan
  shape (leaf chunks of 4, radix-4 folds), and against the FP64 oracle's
  sequential square-root filter and smoother at the tests' tolerances;
- at n = 1, 2, 5 (one chunk per scan level, the single-level paths) and at
  the largest n the fixed scratch admits (FP32, n_x = 5), with n + 1 refused;
- device memory: free memory and the torch allocator's count are unchanged
  across calls once the first call has loaded the library's device code.
This file is collected last on purpose."""
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


def _outputs(n, nx, dt):
    dev = "cuda:0"
    return (torch.empty((n + 1, nx), dtype=dt, device=dev),
            torch.empty((n + 1, nx, nx), dtype=dt, device=dev),
            torch.empty((n + 1, nx), dtype=dt, device=dev),
            torch.empty((n + 1, nx, nx), dtype=dt, device=dev),
            torch.empty(1, dtype=torch.float64, device=dev))


def _noalloc(B, t, n, nx, out=None, strides=None):
    dt = t["y"].dtype
    out = _outputs(n, nx, dt) if out is None else out
    args = []
    for i, k in enumerate(("F", "c", "SQ", "H", "d", "SR")):
        s = t[k][0].numel() if strides is None else strides[i]
        args += [t[k].data_ptr(), s]
    mf, Nf, ms, Ns, ll = out
    rc = B.lib.sqsm_lgssm_smooth_noalloc(
        0 if dt == torch.float32 else 1, nx, t["y"].shape[1], n, *args, t["m0"].data_ptr(),
        t["N0"].data_ptr(), t["y"].data_ptr(), mf.data_ptr(), Nf.data_ptr(), ms.data_ptr(),
        Ns.data_ptr(), ll.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, out


def _host(xs):
    return [x.cpu().numpy() for x in xs]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_matches_same_shape_context_and_oracle(B, prec):
    from oracle.kalman import sqrt_filter_smoother
    dtype = torch.float32 if prec == "f32" else torch.float64
    ctx = B.Context(0, leaf_chunk=4, radix=4)
    tol = TOL[prec]
    cases = ((1, (1, 5, 2)), (2, (2, 5, 2)), (3, (5, 5, 2)), (4, (3000, 5, 2)),
             (5, (777, 4, 2)), (6, (2, 4, 2)))
    for seed, (n, nx, ny) in cases:
        m = W.random_lgssm(n, nx, ny, seed=seed)
        t = _tensors(m, dtype)
        rc, got = _noalloc(B, t, n, nx)
        assert rc == B.OK, (n, nx)
        same = B.sqsm_lgssm_smooth(ctx, t["F"], t["c"], t["SQ"], t["H"], t["d"], t["SR"],
                                   t["m0"], t["N0"], t["y"])
        torch.cuda.synchronize()
        got, same = _host(got), _host(same)
        for g, r in zip(got, same):
            assert np.array_equal(g, r), (n, nx)
        mf, Nf, ms, Ns, ll = sqrt_filter_smoother(m["F"], m["c"], m["SQ"], m["H"], m["d"],
                                                  m["SR"], m["y"], m["m0"], m["N0"])
        assert rel_mean_err(got[0], mf) <= tol["mean"], (n, nx)
        assert rel_mean_err(got[2], ms) <= tol["mean"], (n, nx)
        assert rel_cov_err(got[1], Nf) <= tol["cov"], (n, nx)
        assert rel_cov_err(got[3], Ns) <= tol["cov"], (n, nx)
        assert abs(got[4][0] - ll) <= tol["ll"] * abs(ll), (n, nx)
    ctx.close()


def test_noalloc_allocates_nothing(B):
    n, nx, ny = 4000, 5, 2
    m = W.random_lgssm(n, nx, ny, seed=7)
    t = _tensors(m, torch.float32)
    out = _outputs(n, nx, torch.float32)
    rc, _ = _noalloc(B, t, n, nx, out)      # first call on the device: set-up
    assert rc == B.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    lls = []
    for _ in range(3):
        rc, _ = _noalloc(B, t, n, nx, out)
        assert rc == B.OK
        torch.cuda.synchronize()
        lls.append(out[4].item())
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert lls[0] == lls[1] == lls[2] and np.isfinite(lls[0])


def test_noalloc_largest_admitted_size(B):
    """Bisect the largest n the 32 MiB scratch admits (FP32, n_x = 5, a
    time-invariant model); that call runs and matches the same-shape context
    bit for bit, and n + 1 is refused before any GPU work."""
    nx, ny = 5, 2
    m1 = W.random_lgssm(1, nx, ny, seed=8)
    hi_n = 140_000
    rng = np.random.default_rng(9)
    t = _tensors({k: m1[k][0] if k in ("F", "c", "SQ", "H", "d", "SR") else m1[k]
                  for k in ("F", "c", "SQ", "H", "d", "SR", "m0", "N0")}, torch.float32)
    t["y"] = torch.tensor(rng.standard_normal((hi_n, ny)), dtype=torch.float32, device="cuda:0")
    for k in ("F", "c", "SQ", "H", "d", "SR"):
        t[k] = t[k][None]          # one row, stride 0
    out = _outputs(hi_n, nx, torch.float32)
    zero = (0,) * 6
    lo, hi = 1, hi_n               # rc(lo) == OK, rc(hi) == TOO_LARGE
    rc_hi, _ = _noalloc(B, t, hi, nx, out, zero)
    assert rc_hi == B.ERR_TOO_LARGE
    while hi - lo > 1:
        mid = (lo + hi) // 2
        rc, _ = _noalloc(B, t, mid, nx, out, zero)
        assert rc in (B.OK, B.ERR_TOO_LARGE)
        if rc == B.OK:
            lo = mid
        else:
            hi = mid
    n = lo
    assert n > 100_000
    torch.cuda.synchronize()
    # a small call, then the largest one, then compare with the context path
    rc, _ = _noalloc(B, t, 5, nx, _outputs(5, nx, torch.float32), zero)
    assert rc == B.OK
    outn = _outputs(n, nx, torch.float32)
    rc, got = _noalloc(B, t, n, nx, outn, zero)
    assert rc == B.OK
    ctx = B.Context(0, leaf_chunk=4, radix=4)
    y = t["y"][:n].contiguous()
    same = B.sqsm_lgssm_smooth(ctx, t["F"][0], t["c"][0], t["SQ"][0], t["H"][0], t["d"][0],
                               t["SR"][0], t["m0"], t["N0"], y)
    torch.cuda.synchronize()
    for g, r in zip(_host(got), _host(same)):
        assert np.array_equal(g, r)
    assert np.isfinite(got[4].item())
    ctx.close()
    rc, _ = _noalloc(B, t, n + 1, nx, out, zero)
    assert rc == B.ERR_TOO_LARGE


def test_noalloc_rejects_too_large(B):
    n = 10_000_000
    t = {k: torch.zeros(1, device="cuda:0") for k in ("F", "c", "SQ", "H", "d", "SR", "m0", "N0", "y")}
    p = t["y"].data_ptr()
    rc = B.lib.sqsm_lgssm_smooth_noalloc(0, 5, 2, n, *([p, 0] * 6), p, p, p, p, p, p, p, None,
                                         torch.cuda.current_stream().cuda_stream)
    assert rc == B.ERR_TOO_LARGE
