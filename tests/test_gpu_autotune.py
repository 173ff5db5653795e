"""The scan-shape autotuner: the measured choice is one of the candidates,
is stored per workload shape, and gives the same smoother (within FP32
rounding of a different bracketing) as the default shape."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_00426_gb300 import workloads as W
from gpu_util import rel_mean_err

CANDIDATES = {(2, 0), (3, 0), (4, 0), (6, 0), (8, 0), (4, 4)}


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def test_autotuned_shape_matches_default(B):
    d = W.ct_batch(batch=48, lo=50, hi=700, seed=5)
    tuned = B.Context(0, autotune=True)
    plain = B.Context(0)
    f64 = torch.float64
    args = (d["theta"], _dev(d["y"], f64), d["offsets"], _dev(d["m0"], f64), _dev(d["N0"], f64),
            3, 0)
    assert tuned.scan_shape(d["offsets"], f64) == plain.scan_shape(d["offsets"], f64)
    ms_t, Ns_t, ll_t = B.sqsm_ipls_smooth(tuned, *args, dt=d["dt"])
    ms_p, Ns_p, ll_p = B.sqsm_ipls_smooth(plain, *args, dt=d["dt"])
    torch.cuda.synchronize()
    shape = tuned.scan_shape(d["offsets"], f64)
    assert shape in CANDIDATES
    assert tuned.status() == 0
    # a different bracketing of the same scans: equal up to FP64 rounding
    assert rel_mean_err(ms_t.cpu().numpy(), ms_p.cpu().numpy()) < 1e-9
    np.testing.assert_allclose(ll_t.cpu().numpy(), ll_p.cpu().numpy(), rtol=1e-9)
    # the stored choice is reused (same shape, same result bit for bit)
    ms_2, _, ll_2 = B.sqsm_ipls_smooth(tuned, *args, dt=d["dt"])
    torch.cuda.synchronize()
    assert tuned.scan_shape(d["offsets"], f64) == shape
    assert torch.equal(ms_2, ms_t) and torch.equal(ll_2, ll_t)
    # a different workload shape is not covered by the stored choice
    other = [0, 10, 25]
    assert tuned.scan_shape(other, f64) == plain.scan_shape(other, f64)
    assert tuned.scan_shape(d["offsets"], torch.float32) == plain.scan_shape(d["offsets"])
    tuned.close()
    plain.close()


def test_autotune_off_when_shape_is_given(B):
    c = B.Context(0, leaf_chunk=2, autotune=True)
    d = W.ct_batch(lengths=[40, 7], seed=6)
    B.sqsm_ipls_smooth(c, d["theta"], _dev(d["y"]), d["offsets"], _dev(d["m0"]), _dev(d["N0"]),
                       2, 0, dt=d["dt"])
    torch.cuda.synchronize()
    assert c.scan_shape(d["offsets"]) == (2, 0)
    c.close()


def test_autotuned_gradient(B):
    d = W.ct_batch(lengths=[300, 120, 41], seed=7)
    args = (d["theta"], _dev(d["y"], torch.float64), d["offsets"], _dev(d["m0"], torch.float64),
            _dev(d["N0"], torch.float64))
    tuned = B.Context(0, autotune=True)
    plain = B.Context(0)
    n1, g1, _, _, _ = B.sqsm_ipls_nll_grad(tuned, *args, M=8, adj_iters=8, dt=d["dt"])
    n2, g2, _, _, _ = B.sqsm_ipls_nll_grad(plain, *args, M=8, adj_iters=8, dt=d["dt"])
    torch.cuda.synchronize()
    assert tuned.scan_shape(d["offsets"], torch.float64) in CANDIDATES
    assert abs(n1.item() - n2.item()) <= 1e-10 * abs(n2.item())
    np.testing.assert_allclose(g1.cpu().numpy(), g2.cpu().numpy(), rtol=1e-8, atol=1e-10)
    tuned.close()
    plain.close()
