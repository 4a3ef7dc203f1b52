"""Multi-process trial sharding on CPU (gloo, world size 2): each rank anneals
its own contiguous trial range with global trial indices; the gathered result
equals one run over all trials, and the max-over-ranks timing reduction works.
The per-rank compute here is the oracle (the GPU path shares its keying by
trial index and is checked against the oracle elsewhere)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2302_12454_gb300.sharding import trial_range


def test_trial_range_partitions():
    for total in (0, 1, 7, 64, 1024, 1025):
        for world in (1, 2, 3, 8):
            got = [trial_range(r, world, total) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch

    from oracle import oracle as O
    from paper_2302_12454_gb300.sharding import gather_trials

    a = O.gen_er_graph(5, 1 << 31, 7)
    b, _ = O.permute_graph(a, 8)
    h, J, off = O.build_gi_ising(a, b)
    total = 9
    s0, s1 = trial_range(rank, world, total)
    local = O.anneal(h, J, R=4, cycles=60, trials=max(s1 - s0, 0), seed=5, tau=10, trial_offset=s0) \
        if s1 > s0 else None
    local = {k: v for k, v in local.items()}
    full = gather_trials(local, dist)
    t = torch.tensor([1.0 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.savez(os.path.join(out_dir, "gathered.npz"), **full, tmax=t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_equals_single_run(tmp_path):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    from oracle import oracle as O
    a = O.gen_er_graph(5, 1 << 31, 7)
    b, _ = O.permute_graph(a, 8)
    h, J, off = O.build_gi_ising(a, b)
    ref = O.anneal(h, J, R=4, cycles=60, trials=9, seed=5, tau=10)
    got = np.load(tmp_path / "gathered.npz")
    for k in ("sigma", "Is", "E_final", "hist"):
        np.testing.assert_array_equal(got[k], ref[k])
    assert float(got["tmax"][0]) == 2.0
