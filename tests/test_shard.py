"""Sharding of a cone batch across ranks: world size 2 on gloo (CPU).

Each rank takes its part of the uneven-batch shapes, projects its cones
(here with the FP64 oracle: the test runs without a GPU), and the gathered
output must equal the oracle's projection of the whole batch bit for bit
(the oracle is deterministic cone by cone)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_20519_gb300 import shard
from paper_2606_20519_gb300 import workloads as W


def test_partition_covers_and_balances():
    sides = [4, 9, 16, 25, 36, 49, 64] * 4 + [625, 1296, 625]
    for world in (1, 2, 3, 8):
        parts = shard.partition(sides, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sides)))
        assert all(p == sorted(p) for p in parts)
        loads = [sum(sides[i] ** 3 for i in p) for p in parts]
        # greedy largest-first: no rank exceeds the ideal share by more than the largest cone
        assert max(loads) <= sum(loads) / world + max(s ** 3 for s in sides)
    assert shard.partition(sides, 2) == shard.partition(list(sides), 2)  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, x, sides, q):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = shard.partition(sides, world)
        xl, sl = shard.pack(torch.from_numpy(x), sides, parts[rank])
        yl = oracle.proj_batched(xl.numpy(), shard.offsets_of(sl)) if sl else np.zeros(0)
        y = shard.gather(torch.from_numpy(np.ascontiguousarray(yl)), sides, parts)
        if rank == 0:
            q.put(y.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_shard_and_gather():
    import oracle
    oracle.build()
    sides = [4, 9, 16, 1, 25, 36, 40, 9, 16, 2]
    rng = W.rng_for(777)
    x = np.concatenate([W.to_svec(W.sym_gaussian(rng, n)) for n in sides])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, x, sides, q)) for r in range(2)]
    for p in procs:
        p.start()
    y = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = oracle.proj_batched(x, shard.offsets_of(sides))
    assert np.array_equal(y, ref)
