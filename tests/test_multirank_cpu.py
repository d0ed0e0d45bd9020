"""Multi-rank paths on the CPU (gloo, world size 2), no GPU.

1. The one sharding of a single tree the method allows: G contiguous
   subtrees built apart, their roots gathered to rank 0, which hashes the top
   log2(G) levels (Sec. 4.2's level-by-level rule).  The gathered root must
   equal the root of the whole tree.
2. The replica pattern bench.py uses for N GPUs: every rank builds its own
   tree, the step time is the maximum over ranks, and throughput counts the
   work of all ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import pg_synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, w, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rows = pg_synth.matrix(0x5EED0077, n, w)
        part = n // world
        sub = oracle.merkle_build(rows[rank * part:(rank + 1) * part])
        root = torch.from_numpy(sub[-1].view(np.int64).copy())
        gathered = [torch.zeros(4, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(gathered, root)
        # replica timing pattern: max over ranks
        t = torch.tensor([float(rank + 1)])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            level = [g.numpy().view(np.uint64) for g in gathered]
            while len(level) > 1:
                level = [oracle.hash_pair(level[2 * i], level[2 * i + 1]) for i in range(len(level) // 2)]
            q.put(([int(v) for v in level[0]], float(t.item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_subtree_split_gather_equals_full_root(world):
    n, w = 64, 8
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, w, q)) for r in range(world)]
    for p in procs:
        p.start()
    root, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    full = oracle.merkle_build(pg_synth.matrix(0x5EED0077, n, w))
    assert root == [int(v) for v in full[-1]]
    assert tmax == float(world)
