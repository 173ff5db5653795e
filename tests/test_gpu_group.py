"""NLL + gradient with a bounded workspace (sqsm_options.max_group_steps):
a batch evaluated in groups of consecutive sequences gives the NLL, the
gradient and the trajectory of the whole-batch call (sums over independent
sequences), frees each group's workspace, refuses a sequence longer than the
bound, and reports the larger of the groups' changes; the workspace per time
step that the bound is stated in is measured."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_00426_gb300 import workloads as W

LENGTHS = [300, 420, 250, 380, 500, 310]   # groups at 800: [300 420] [250 380] [500] [310]


@pytest.fixture(scope="module")
def B():
    from paper_2207_00426_gb300 import binding
    return binding


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _eval(B, ctx, d, dtype, M=8, adj=8, tol=0.0):
    y, m0, N0 = (_dev(d[k], dtype) for k in ("y", "m0", "N0"))
    ich = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    nll, g, ch, ms, Ns = B.sqsm_ipls_nll_grad(ctx, d["theta"], y, d["offsets"], m0, N0, M, adj,
                                              dt=d["dt"], tol=tol, ipls_change=ich)
    torch.cuda.synchronize()
    return (nll.item(), g.cpu().numpy(), ch.item(), ich.item(), ms.double().cpu().numpy(),
            Ns.double().cpu().numpy())


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 2e-5)])
def test_grouped_equals_whole_batch(B, dtype, tol):
    d = W.ct_batch(lengths=LENGTHS, seed=21)
    whole = B.Context(0)
    grouped = B.Context(0, max_group_steps=800)
    nw, gw, cw, iw, msw, Nsw = _eval(B, whole, d, dtype)
    ng, gg, cg, ig, msg, Nsg = _eval(B, grouped, d, dtype)
    assert abs(ng - nw) <= tol * abs(nw)
    assert np.max(np.abs(gg - gw)) <= 10 * tol * np.max(np.abs(gw))
    assert np.max(np.abs(msg - msw)) <= 10 * tol * np.max(np.abs(msw))
    assert np.max(np.abs(Nsg - Nsw)) <= 10 * tol * np.max(np.abs(Nsw)) + 10 * tol
    # each group's change is relative to its own max-norm: never below the
    # whole batch's
    slack = 1e-6 if dtype == torch.float64 else 1e-2
    assert cg >= cw * (1 - slack) and ig >= iw * (1 - slack)
    assert whole.status() == 0 and grouped.status() == 0
    whole.close()
    grouped.close()


def _outputs(n_steps, batch, dtype):
    rows = n_steps + batch
    return dict(ms=torch.empty((rows, 5), dtype=dtype, device="cuda:0"),
                Ns=torch.empty((rows, 5, 5), dtype=dtype, device="cuda:0"),
                nll=torch.empty(1, dtype=torch.float64, device="cuda:0"),
                grad=torch.empty(3, dtype=torch.float64, device="cuda:0"),
                change=torch.empty(1, dtype=torch.float64, device="cuda:0"))


def test_grouped_call_frees_its_workspace(B):
    d = W.ct_batch(lengths=[20000] * 6, seed=22)
    f32 = torch.float32
    y, m0, N0 = (_dev(d[k], f32) for k in ("y", "m0", "N0"))
    out = _outputs(d["y"].shape[0], 6, f32)
    torch.cuda.synchronize()
    ctx = B.Context(0, use_graph=False, max_group_steps=40000)
    free0 = torch.cuda.mem_get_info()[0]
    B.sqsm_ipls_nll_grad(ctx, d["theta"], y, d["offsets"], m0, N0, 2, 2, dt=d["dt"], **out)
    torch.cuda.synchronize()
    # every group's plan and workspace (about 150 MB each) are gone again
    assert free0 - torch.cuda.mem_get_info()[0] <= 8 * 2**20
    assert ctx.status() == 0
    ctx.close()


def test_workspace_per_step_as_stated(B):
    """The bound is stated as about 3.4 KB per step (FP32) and 6.6 KB
    (FP64): the first whole-batch call's allocation on 120000 steps."""
    d = W.ct_batch(lengths=[40000] * 3, seed=23)
    per_step = {}
    for dtype, es in ((torch.float32, 4), (torch.float64, 8)):
        y, m0, N0 = (_dev(d[k], dtype) for k in ("y", "m0", "N0"))
        n = d["y"].shape[0]
        out = _outputs(n, 3, dtype)
        torch.cuda.synchronize()
        ctx = B.Context(0, use_graph=False)
        free0 = torch.cuda.mem_get_info()[0]
        B.sqsm_ipls_nll_grad(ctx, d["theta"], y, d["offsets"], m0, N0, 1, 1, dt=d["dt"], **out)
        torch.cuda.synchronize()
        per_step[es] = (free0 - torch.cuda.mem_get_info()[0]) / n
        ctx.close()
    print("workspace bytes per step", per_step)
    assert 2500 <= per_step[4] <= 4500, per_step
    assert 5000 <= per_step[8] <= 9000, per_step


def test_sequence_longer_than_the_bound_is_refused(B):
    d = W.ct_batch(lengths=[300, 900], seed=24)
    ctx = B.Context(0, max_group_steps=800)
    with pytest.raises(B.SqsmError) as e:
        _eval(B, ctx, d, torch.float64)
    assert e.value.code == B.ERR_TOO_LARGE
    ctx.close()


def test_grouped_fixed_point_check(B):
    """tol: a group that has not settled sets SQSM_ERR_NOT_CONVERGED."""
    d = W.ct_batch(lengths=LENGTHS, seed=21)
    ctx = B.Context(0, max_group_steps=800)
    _eval(B, ctx, d, torch.float64, M=1, adj=2, tol=1e-6)
    assert ctx.status() == B.ERR_NOT_CONVERGED
    ctx.close()
