"""torch.autograd.Function for the negative pseudo log-likelihood of the CT
bearings model as a function of theta = (log sigma, log q_c, log q_omega),
or of theta = (log sqrt(R_11), log q_c, log q_omega, log sqrt(R_22)) with
one noise level per sensor (Sec. 6.4).

forward() calls sqsm_ipls_nll_grad (IPLS to the trajectory n*, the
pseudo log-likelihood of Sec. 5.1 and its gradient by the hand-written
adjoint of Sec. 5.2) and keeps the gradient; backward() scales it by the
incoming gradient.  theta is a CPU float64 tensor of shape (3,) or (4,)
(the C ABI takes the parameters on the host); the data live on the GPU.
"""
import torch

from . import binding as B


class IplsNLL(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, ctx, y, offsets, m0, N0, M, adj_iters, dt):
        th = theta.detach().cpu().double().tolist()
        nll, grad, change, _, _ = B.sqsm_ipls_nll_grad(ctx, th, y, offsets, m0, N0, M, adj_iters,
                                                       dt=dt)
        fctx.save_for_backward(grad.detach().cpu())
        return nll.detach().cpu().reshape(())

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return (g * grad, None, None, None, None, None, None, None, None)


def ipls_nll(theta, ctx, y, offsets, m0, N0, M=10, adj_iters=20, dt=0.01):
    """Negative pseudo log-likelihood (summed over the batch), differentiable
    in theta through the implicit-function adjoint."""
    return IplsNLL.apply(theta, ctx, y, offsets, m0, N0, M, adj_iters, dt)
