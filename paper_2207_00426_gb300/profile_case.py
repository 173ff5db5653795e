"""One IPLS solve of a benchmark workload, for profiling the kernels with a
fixed, reproducible launch sequence (ncu -k / -s / -c select from it).

  python -m paper_2207_00426_gb300.profile_case single --n 100000 --M 2
  python -m paper_2207_00426_gb300.profile_case batch --batch 1024 --M 1
  python -m paper_2207_00426_gb300.profile_case grad --n 100000 --M 2 --adj 2

single  one coordinated-turn sequence (seed 1), cubature IPLS
batch   CT sequences with lengths U{100..5000} (seed 3, the first --batch of
        the 4096-sequence workload's draw)
grad    NLL + gradient of one sequence
Graphs are off (each kernel is its own launch) unless --graph; --reps
repeats the call (the first call builds plans and workspaces).
"""
import argparse
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["single", "batch", "grad"])
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--M", type=int, default=2)
    ap.add_argument("--adj", type=int, default=2)
    ap.add_argument("--f64", action="store_true")
    ap.add_argument("--leaf", type=int, default=0)
    ap.add_argument("--refine", type=int, default=0)
    ap.add_argument("--graph", action="store_true")
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args(argv)
    import torch
    from . import binding as B
    from . import workloads as W
    dt = torch.float64 if a.f64 else torch.float32
    T = lambda v: torch.tensor(np.ascontiguousarray(v), dtype=dt, device="cuda:0")
    ctx = B.Context(0, use_graph=a.graph, leaf_chunk=a.leaf, refine=a.refine)
    if a.case == "batch":
        full = W.ct_batch(batch=4096, lo=100, hi=5000, seed=3)
        off = [int(v) for v in full["offsets"][:a.batch + 1]]
        d = dict(full, y=full["y"][:off[-1]], m0=full["m0"][:a.batch], N0=full["N0"][:a.batch])
    else:
        d = W.ct_sequence(n=a.n, seed=1)
        d = dict(d, m0=d["m0"][None], N0=d["N0"][None])
        off = [0, a.n]
    y, m0, N0 = T(d["y"]), T(d["m0"]), T(d["N0"])
    for _ in range(a.reps):
        if a.case == "grad":
            B.sqsm_ipls_nll_grad(ctx, d["theta"], y, off, m0, N0, a.M, a.adj, dt=d["dt"])
        else:
            B.sqsm_ipls_smooth(ctx, d["theta"], y, off, m0, N0, a.M, dt=d["dt"])
    torch.cuda.synchronize()
    st = ctx.status()
    ctx.close()
    if st != 0:
        print(f"device status {st}", file=sys.stderr)
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
