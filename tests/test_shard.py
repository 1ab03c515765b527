"""Multi-GPU host logic on CPU: beams shard across ranks with no data exchange.

Two gloo ranks each compute their share of a batch of beams; gathering the
shares shows every beam is assigned exactly once and the load is balanced.
The max-over-ranks timing reduction the benchmark uses is checked too."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1601_01165_gb300 import synth
from paper_1601_01165_gb300.shard import beam_cost, rank_beams, shard_beams


def test_shard_covers_each_beam_once():
    costs = [beam_cost(s) for s, _ in synth.batched_setups(0)]
    for world in (1, 2, 3, 8):
        parts = shard_beams(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)        # LPT bound


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    costs = [beam_cost(s) for s, _ in synth.batched_setups(0)]
    mine = rank_beams(costs, world, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)      # the benchmark's max-over-ranks time
    q.put((rank, gathered, float(t)))
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_beams():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, tmax in res:
        assert tmax == 2.0
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(64))
        assert not set(gathered[0]) & set(gathered[1])
