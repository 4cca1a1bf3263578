"""The N > 1 path on CPU: independent TMCMC runs on two `gloo` ranks, no data-path
collective, and the measurement's SUM / MAX reductions.  Each rank runs the oracle's TMCMC
on the Gaussian toy posterior (closed form N(mean, sd^2)) with its own seed; the pooled
samples of both ranks must match the closed form, and the two runs must differ."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import synthetic  # noqa: E402
from paper_1910_12007_gb300 import ranks  # noqa: E402

MEAN = np.array([0.7, -1.2, 2.0])
SD = np.array([0.3, 0.5, 0.2])
B = 1024


def _loglik(th):
    th = np.atleast_2d(th)
    return -0.5 * np.sum(((th - MEAN) / SD) ** 2, axis=1)


def _worker(rank, world, port, outdir):
    from oracle import tmcmc as tm

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, _ = ranks.rank_env()
    tdist.init_process_group("gloo", rank=r, world_size=w)
    seed = ranks.rank_seed(11, r)
    lo, hi = np.full(3, -8.0), np.full(3, 8.0)
    th0 = synthetic.prior_samples(seed, lo, hi, B)
    theta, _, log = tm.run(th0, _loglik, lo, hi, seed, randoms=lambda j: synthetic.stage_randoms(seed, j, B, 3))
    # measurement reductions: work summed, time maxed
    sums, maxes = ranks.totals(tdist, [B, len(log.q)], [float(r + 1)])
    tdist.barrier()
    np.savez(os.path.join(outdir, f"rank{r}.npz"), theta=theta, sums=np.array(sums), maxes=np.array(maxes),
             stages=len(log.q))
    tdist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_partitions_units():
    for total in (0, 1, 5, 1024, 4097):
        for world in range(1, 9):
            parts = [ranks.shard(total, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == total
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ranks.shard(10, 2, 2)


def test_rank_seeds_give_independent_inputs():
    assert ranks.rank_seed(1000, 0) == 1000
    a = synthetic.prior_samples(ranks.rank_seed(1000, 0), (0, -1, 0.05), (10, 1, 0.2), 64)
    b = synthetic.prior_samples(ranks.rank_seed(1000, 1), (0, -1, 0.05), (10, 1, 0.2), 64)
    assert not np.array_equal(a, b)


def test_totals_without_process_group():
    assert ranks.totals(None, [3, 4], [5]) == ([3.0, 4.0], [5.0])


def test_two_gloo_ranks_run_independent_tmcmc():
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(2, port, d), nprocs=2, join=True)
        res = [np.load(os.path.join(d, f"rank{r}.npz")) for r in range(2)]
    # SUM of work over ranks, MAX of time, identical on every rank
    for r in res:
        assert r["sums"][0] == 2 * B
        assert r["sums"][1] == res[0]["stages"] + res[1]["stages"]
        assert r["maxes"][0] == 2.0
    t0, t1 = res[0]["theta"], res[1]["theta"]
    assert not np.allclose(t0, t1)  # independent runs
    pooled = np.concatenate([t0, t1])
    # pooled 2048 samples: the closed-form posterior within 3 Monte-Carlo standard errors
    assert np.all(np.abs(pooled.mean(0) - MEAN) < 0.3 * SD)
    assert np.all(np.abs(pooled.std(0) / SD - 1) < 0.1)
