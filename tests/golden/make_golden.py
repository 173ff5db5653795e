"""Writes the stored expected values of the full-size parity tests.

Calls only the FP64 oracle (oracle/) and the seeded workload generator
(paper_2207_00426_gb300/workloads.py, random draws and model simulation
only); nothing here touches the CUDA path.  Each file records the workload,
the oracle call that produced it and a checksum of the generated inputs, so
a test can tell a drifted generator from a wrong kernel.

  python tests/golden/make_golden.py ipls     # ~10 min, one core
  python tests/golden/make_golden.py frozen   # ~2 min, 7 processes

ipls   -> ipls_ct_n1e5_seed1_M10.npz: Alg. 3 (cubature, M = 10, prior
          broadcast as the initial trajectory) on the n = 1e5 coordinated-turn
          sequence of seed 1: smoothed means of every 20th state row, lower
          factors of every 200th, and the pseudo log-likelihood (Sec. 5.1).
frozen -> frozen_grad_ct_n1e5_seed1.json: the pseudo log-likelihood of the
          cubature linearisation (Sec. 4.3) about a fixed trajectory -- the
          simulated true states with the factor 0.05 I at every step -- and
          its derivative in theta, the partial gradient of Sec. 5.2 at a
          frozen trajectory.  The derivative is Richardson's extrapolation
          of central differences at h = 1e-4 and h / 2,
          (4 D(h/2) - D(h)) / 3: a plain central difference carries the
          truncation error h^2 / 6 times the third derivative, which here
          is ~1.3e-3 in d/d log sigma (the sum of 2e5 bearing terms has a
          third derivative of ~8e5), far above the FP64 kernels' error.
"""
import json
import os
import sys

# one BLAS thread per process: the oracle works on 5 x 10 blocks, where
# threading only adds overhead (the frozen-trajectory file runs 7 processes)
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N = 100_000
SEED = 1
M = 10
MEAN_EVERY = 20
FACTOR_EVERY = 200
FROZEN_FACTOR = 0.05
H = 1e-4


def checksum(a):
    return float(np.sum(np.asarray(a, dtype=np.float64) * np.arange(1, a.size + 1).reshape(a.shape)
                        / a.size))


def make_ipls():
    from oracle import ipls as O, models as OM
    from paper_2207_00426_gb300 import workloads as W
    d = W.ct_sequence(n=N, seed=SEED)
    ct = OM.CTBearings(d["theta"], dt=d["dt"])
    ms, Ns, ll, _ = O.ipls(ct, d["y"], d["m0"], d["N0"], M, "cubature")
    rows_m = np.arange(0, N + 1, MEAN_EVERY)
    rows_N = np.arange(0, N + 1, FACTOR_EVERY)
    np.savez_compressed(os.path.join(HERE, "ipls_ct_n1e5_seed1_M10.npz"),
                        rows_m=rows_m, ms=ms[rows_m], rows_N=rows_N, Ns=Ns[rows_N],
                        loglik=np.float64(ll), n=N, seed=SEED, M=M,
                        y_checksum=checksum(d["y"]))


def _frozen_ll(theta):
    from oracle import kalman as K, models as OM, slr as S
    from paper_2207_00426_gb300 import workloads as W
    d = W.ct_sequence(n=N, seed=SEED)
    ct = OM.CTBearings(theta, dt=d["dt"])
    ms = d["x"]
    Ns = np.tile(FROZEN_FACTOR * np.eye(5), (N + 1, 1, 1))
    G = S.linearize(ct, ms, Ns, d["y"], "cubature")
    _, _, ell = K.sqrt_filter(*G, d["y"], d["m0"], d["N0"])
    return float(np.sum(ell))


def make_frozen():
    import multiprocessing as mp
    from paper_2207_00426_gb300 import workloads as W
    d = W.ct_sequence(n=N, seed=SEED)
    th = np.asarray(d["theta"], dtype=np.float64)
    pts = [th]
    for step in (H, H / 2):
        for j in range(th.size):
            for sgn in (1.0, -1.0):
                t = th.copy()
                t[j] += sgn * step
                pts.append(t)
    with mp.get_context("spawn").Pool(min(len(pts), os.cpu_count() or 1)) as pool:
        lls = pool.map(_frozen_ll, pts)
    k = th.size

    def central(i, half):
        base = 1 + (2 * k if half else 0)
        step = H / 2 if half else H
        return -(lls[base + 2 * i] - lls[base + 2 * i + 1]) / (2 * step)
    d1 = [central(i, False) for i in range(k)]
    d2 = [central(i, True) for i in range(k)]
    grad = [(4 * b - a) / 3 for a, b in zip(d1, d2)]
    out = {"workload": f"CT bearings, n={N}, seed={SEED}", "theta": th.tolist(), "h": H,
           "trajectory": f"simulated true states, factor {FROZEN_FACTOR} I at every step",
           "linearization": "cubature", "nll": -lls[0], "grad_nll": grad,
           "derivative": "Richardson: (4 D(h/2) - D(h)) / 3 of central differences D",
           "central_h": d1, "central_h_half": d2,
           "x_checksum": checksum(d["x"]), "y_checksum": checksum(d["y"])}
    with open(os.path.join(HERE, "frozen_grad_ct_n1e5_seed1.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    what = sys.argv[1:] or ["frozen", "ipls"]
    for w in what:
        {"ipls": make_ipls, "frozen": make_frozen}[w]()
