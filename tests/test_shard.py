"""Multi-GPU host logic on CPU: beams shard across ranks with no data exchange.

Two gloo ranks each compute their share of a batch of beams and their block
of one beam's DM trials; gathering the shares shows every beam and every
trial is assigned exactly once and the load is balanced.  The max-over-ranks
timing reduction the benchmark uses is checked too."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1601_01165_gb300 import synth
from paper_1601_01165_gb300.shard import beam_cost, rank_beams, shard_beams, split_dm_range


def test_shard_covers_each_beam_once():
    costs = [beam_cost(s) for s, _ in synth.batched_setups(0)]
    for world in (1, 2, 3, 8):
        parts = shard_beams(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)        # LPT bound


@pytest.mark.parametrize("n_dm,world,align", [(2048, 1, 6), (2048, 2, 6), (2048, 3, 6), (2048, 8, 64),
                                             (4096, 7, 8), (13, 4, 6), (5, 8, 1), (1, 3, 6), (0, 2, 6)])
def test_split_dm_range_covers_each_trial_once(n_dm, world, align):
    parts = split_dm_range(n_dm, world, align)
    assert len(parts) == world
    assert parts[0][0] == 0 and parts[-1][1] == n_dm
    for (a0, a1), (b0, b1) in zip(parts, parts[1:]):
        assert a1 == b0                                   # contiguous, no overlap
    sizes = [i1 - i0 for i0, i1 in parts]
    assert all(s >= 0 for s in sizes) and sum(sizes) == n_dm
    assert all(i0 % align == 0 for i0, i1 in parts if i0 < n_dm)   # blocks start on a kernel tile
    full = [s for s in sizes if s > 0][:-1]               # all but the last non-empty block are whole units
    assert all(s % align == 0 for s in full)
    assert max(sizes) - min(sizes) <= align or n_dm < world * align


def test_split_dm_range_rejects_bad_arguments():
    for args in ((10, 0, 1), (10, 2, 0), (-1, 2, 1)):
        with pytest.raises(ValueError):
            split_dm_range(*args)


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
    mine = (rank_beams(costs, world, rank), split_dm_range(synth.APERTIF.n_dm, world, 6)[rank])
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
        beams = [g[0] for g in gathered]
        flat = sorted(i for part in beams for i in part)
        assert flat == list(range(64))
        assert not set(beams[0]) & set(beams[1])
        # one beam split by DM trials: the two ranks' blocks tile [0, n_dm)
        (a0, a1), (b0, b1) = gathered[0][1], gathered[1][1]
        assert a0 == 0 and a1 == b0 and b1 == synth.APERTIF.n_dm
