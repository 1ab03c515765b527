"""Sharding beams across GPUs (one process per GPU).

Beams are independent (Section 2), so N GPUs split a set of beams with no
data exchange: each beam goes to exactly one rank, largest first onto the
least-loaded rank (longest-processing-time order), where a beam's cost is
channels x DM trials x output samples (Algorithm 1's d x s x c).
"""
from __future__ import annotations


def beam_cost(setup) -> int:
    return int(setup.channels) * int(setup.n_dm) * int(setup.n_out)


def shard_beams(costs, world_size: int) -> list[list[int]]:
    """Assign beam indices to ranks: returns one list of beam indices per rank."""
    if world_size <= 0:
        raise ValueError("world_size must be positive")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world_size
    out: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return out


def rank_beams(costs, world_size: int, rank: int) -> list[int]:
    return shard_beams(costs, world_size)[rank]
