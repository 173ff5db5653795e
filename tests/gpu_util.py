"""Helpers of the GPU parity tests: error metrics against the oracle."""
import numpy as np


def rel_mean_err(m, ref):
    """max_k |m_k - ref_k|_2 / max_k |ref_k|_2"""
    return np.linalg.norm(m - ref, axis=-1).max() / max(np.linalg.norm(ref, axis=-1).max(), 1e-300)


def rel_cov_err(N, Nref):
    """max_k |N N^T - Nr Nr^T|_F / max_k |Nr Nr^T|_F"""
    P = N @ np.swapaxes(N, -1, -2)
    Pr = Nref @ np.swapaxes(Nref, -1, -2)
    return (np.linalg.norm(P - Pr, axis=(-2, -1)).max()
            / max(np.linalg.norm(Pr, axis=(-2, -1)).max(), 1e-300))


# Tolerances: FP32 means 1e-4, log-likelihood 1e-5 relative; FP64 near
# round-off of the sequential oracle.
TOL = {"f32": dict(mean=1e-4, cov=1e-4, ll=1e-5), "f64": dict(mean=1e-9, cov=1e-9, ll=1e-10)}
