"""The multi-GPU host path on CPU: two gloo ranks shard a ragged batch of
sequences, each smooths its shard (here with the FP64 oracle, standing in
for one GPU per rank), and the summed log-likelihood and the max-over-ranks
timing equal the single-process results."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2207_00426_gb300 import dist as D
from paper_2207_00426_gb300 import workloads as W


def test_shard_balances_and_covers():
    rng = np.random.default_rng(0)
    lengths = rng.integers(100, 5000, size=4096)
    for world in (1, 2, 3, 8):
        parts = D.shard_sequences(lengths, world)
        allidx = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(allidx, np.arange(len(lengths)))
        loads = [lengths[p].sum() for p in parts]
        assert max(loads) - min(loads) <= lengths.max()


def test_shard_offsets_and_rows():
    d = W.ct_batch(lengths=[5, 1, 7, 3], seed=2)
    lengths = np.diff(d["offsets"])
    idx = np.array([0, 2])
    off = D.shard_offsets(lengths, idx)
    np.testing.assert_array_equal(off, [0, 5, 12])
    rows = D.gather_rows(d["y"], d["offsets"], idx)
    np.testing.assert_array_equal(rows[:5], d["y"][0:5])
    np.testing.assert_array_equal(rows[5:], d["y"][6:13])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from oracle import ipls as O, models as OM
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = W.ct_batch(lengths=[9, 4, 13, 6, 2], seed=5)
    lengths = np.diff(d["offsets"])
    mine = D.shard_sequences(lengths, world)[rank]
    ll = 0.0
    for b in mine:
        ct = OM.CTBearings(d["theta"], dt=d["dt"])
        yb = d["y"][d["offsets"][b]:d["offsets"][b + 1]]
        _, _, l, _ = O.ipls(ct, yb, d["m0"][b], d["N0"][b], 3, "cubature")
        ll += l
    tot = D.allreduce_sum([ll])[0]
    mx = D.allreduce_max(float(rank + 1))
    out[rank] = (tot, mx, len(mine))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_and_max():
    from oracle import ipls as O, models as OM
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    d = W.ct_batch(lengths=[9, 4, 13, 6, 2], seed=5)
    ref = 0.0
    for b in range(5):
        ct = OM.CTBearings(d["theta"], dt=d["dt"])
        yb = d["y"][d["offsets"][b]:d["offsets"][b + 1]]
        ref += O.ipls(ct, yb, d["m0"][b], d["N0"][b], 3, "cubature")[2]
    for r in range(2):
        tot, mx, cnt = out[r]
        assert abs(tot - ref) < 1e-9 * abs(ref)
        assert mx == 2.0
    assert out[0][2] + out[1][2] == 5
