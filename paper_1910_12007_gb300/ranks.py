"""One process per GPU.

Two ways to use N GPUs:

* independent problems (weak scaling, the default): every rank runs its own TMCMC (or batch
  of forward runs) from its own seeded inputs.  The only collectives belong to a
  measurement: a barrier around the timed region, the SUM of the work done and the MAX of
  the elapsed time over ranks.
* one population sharded over ranks (Sec. 3.2: the samples of a stage are independent):
  every rank holds the same TMCMC state and random numbers and runs the same analysis and
  resampling; the Metropolis chains are split into contiguous blocks of output rows
  balanced by chain length (``chain_owner``), and one SUM all-reduce per stage assembles
  the population (``assemble_stage``; rows of other ranks' chains are zero).
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


def chain_owner(counts, world: int):
    """Owning rank of every chain of a stage, the rule the device applies: chains in
    ascending sample order (samples with counts[k] > 0; chain k's output rows are
    off_k .. off_k + counts[k] - 1, off the exclusive prefix of counts) go to rank
    floor((2 off_k + counts[k]) world / (2 B)), B = sum(counts).  Returns {sample k: rank}."""
    counts = [int(c) for c in counts]
    B = sum(counts)
    out, off = {}, 0
    for k, n in enumerate(counts):
        if n > 0:
            out[k] = ((2 * off + n) * world) // (2 * B)
        off += n
    return out


def assemble_stage(dist, st, use_surrogate=False):
    """After ``tmcmc_stage(..., rank, world)`` on every rank: SUM the per-rank rows of
    st.theta, st.loglik (and st.surr_loglik) into the whole population, and the work
    counters into job totals.  The stage's scalars (q, evidence, covariance) are already
    identical on every rank."""
    if dist is None:
        return st
    tensors = [st.theta, st.loglik] + ([st.surr_loglik] if use_surrogate and st.surr_loglik is not None else [])
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    import torch

    c = st.c
    cnt = torch.tensor([c.n_accept, c.n_exact, c.n_screened, c.n_exact_path], dtype=torch.float64,
                       device=st.theta.device)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    c.n_accept, c.n_exact, c.n_screened, c.n_exact_path = (int(v) for v in cnt.tolist())
    return st
