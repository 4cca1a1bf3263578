"""One process per GPU for work that shards without any exchange.

Every unit of the path is independent (a TMCMC run, a batch of forward runs), so N GPUs run
N independent problems (weak scaling): each rank draws its own seeded inputs and steps its
own handle.  The only collectives belong to a measurement: a barrier around the timed
region, the SUM of the work done and the MAX of the elapsed time over ranks.
"""
from __future__ import annotations

import os

SEED_STRIDE = 100003  # seeds of different ranks never coincide for runs shorter than this


def rank_env():
    """(rank, world size, local rank) from the launcher's environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's independent run; rank 0 keeps `base`."""
    return int(base) + SEED_STRIDE * int(rank)


def shard(total: int, world: int, rank: int):
    """[start, stop) of rank's contiguous share of `total` independent units; shares differ
    by at most one unit."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError(f"bad shard request total={total} world={world} rank={rank}")
    q, r = divmod(total, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def totals(dist, sums, maxes, device=None):
    """All-reduce one measurement over ranks: SUM of `sums` (work), MAX of `maxes` (time).
    `dist` is torch.distributed with an initialized group, or None for a single process."""
    import torch

    s = torch.tensor([float(v) for v in sums], dtype=torch.float64, device=device)
    m = torch.tensor([float(v) for v in maxes], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(s, op=dist.ReduceOp.SUM)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return s.tolist(), m.tolist()
