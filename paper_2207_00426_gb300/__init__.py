"""Parallel square-root smoothers (arXiv 2207.00426) on GB300.

The compute path lives in the CUDA library ``libsqsm.so`` (sources under
``csrc/``, C ABI in ``include/sqsm.h``).  ``binding`` marshals arguments to
it; nothing in this package computes the method on the CPU.  Submodules are
imported explicitly (``from paper_2207_00426_gb300 import binding``), so that
``workloads`` can be used on a machine without a GPU.

Typical use (build once with ``python -m paper_2207_00426_gb300.build``)::

    import torch
    from paper_2207_00426_gb300 import binding as B, workloads as W
    d = W.ct_sequence(n=10_000, seed=1)          # CT bearings-only track
    T = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    ctx = B.Context(0)
    # Alg. 3, M = 10 iterations, cubature SLR: smoothed means, lower
    # covariance factors and the pseudo log-likelihood (Sec. 5.1)
    ms, Ns, ll = B.sqsm_ipls_smooth(ctx, d["theta"], T(d["y"]), [0, 10_000],
                                    T(d["m0"][None]), T(d["N0"][None]), M=10)
    # its negative and the gradient in theta (Sec. 5.2)
    nll, grad, change, _, _ = B.sqsm_ipls_nll_grad(
        ctx, d["theta"], T(d["y"]), [0, 10_000], T(d["m0"][None]),
        T(d["N0"][None]), M=10, adj_iters=10)

Batches of ragged sequences pass their offsets instead of ``[0, n]``;
``autograd.ipls_nll`` wraps the gradient as a ``torch.autograd.Function``.
"""
