"""The multi-GPU form is replicas only (instances never exchange data): every
rank solves its own instance and the job's time is the slowest rank's.  This
checks that host logic of bench.py with two CPU ranks over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = bench.WORKLOADS["c2"]
        seed = bench.replica_seed(w, rank)
        slowest = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, device="cpu")
        specs = bench.batch_specs(bench.WORKLOADS["c4"], rank)
        seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(seeds, torch.tensor([seed]))
        firsts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(firsts, torch.tensor([specs[0][2]]))
        out[rank] = (seed, slowest, [int(t) for t in seeds], [int(t) for t in firsts], len(specs))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] != r1[0] and {r0[0], r1[0]} == {0, 1}        # one instance per rank
    assert r0[1] == r1[1] == 15.0                               # max over ranks on every rank
    assert r0[2] == r1[2] == [0, 1]
    assert r0[3][0] != r0[3][1] and r0[4] == r1[4] == 256       # batch replicas: disjoint seeds
