"""Multi-rank host logic on CPU (gloo, world size 2).

The path shards by stream: each rank creates its own streams from a disjoint
seed range and only the timing is reduced (maximum over ranks).  This checks
the seed partition and the reduction with two real processes, and that the
ranks' streams are independent (different first values from the oracle).
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.rank_seeds(rank, 8)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    t = bench.max_over_ranks(1.5 + rank, world, "cpu")
    first = float(oracle.Stream(64, 2, seeds[0]).generate(1)[0])
    firsts = [None] * world
    dist.all_gather_object(firsts, first)
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        q.put((gathered, t, firsts))


def test_two_ranks_shard_seeds_and_reduce_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t, firsts = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s0, s1 = gathered
    assert len(set(s0) | set(s1)) == 16 and not set(s0) & set(s1)
    assert s0 == list(range(1, 9)) and s1 == list(range(9, 17))
    assert t == 2.5
    assert firsts[0] != firsts[1]
