"""Sharding beams across GPUs (one process per GPU).

Beams are independent (Section 2), so N GPUs split a set of beams with no
data exchange: each beam goes to exactly one rank, largest first onto the
least-loaded rank (longest-processing-time order), where a beam's cost is
channels x DM trials x output samples (Algorithm 1's d x s x c).

One large beam splits by DM trials instead: every DM trial is its own sum
over the channels (Algorithm 1), so rank r takes a contiguous block of
trials (split_dm_range), builds the plan of that block (Plan.dm_range, whose
rows equal the full plan's bit for bit), reads the whole input and writes its
own output rows.  Nothing is exchanged or reduced.
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


def split_dm_range(n_dm: int, world_size: int, align: int = 1) -> list[tuple[int, int]]:
    """Contiguous DM-trial blocks [i0, i1), one per rank, covering [0, n_dm)
    once.  Interior boundaries are multiples of `align` (a kernel's trials per
    block, so no block straddles two ranks); the blocks differ by at most one
    `align` unit.  Ranks past the last unit get empty blocks (i0 == i1)."""
    if world_size <= 0 or align <= 0 or n_dm < 0:
        raise ValueError("world_size and align must be positive, n_dm non-negative")
    units = -(-n_dm // align)
    base, extra = divmod(units, world_size)
    out, u = [], 0
    for r in range(world_size):
        k = base + (1 if r < extra else 0)
        i0, i1 = min(u * align, n_dm), min((u + k) * align, n_dm)
        out.append((i0, i1))
        u += k
    return out
