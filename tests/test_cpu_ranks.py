"""The N > 1 paths on CPU with `gloo` ranks.

Independent runs: each rank runs the oracle's TMCMC on the Gaussian toy posterior (closed
form N(mean, sd^2)) with its own seed; the pooled samples must match the closed form, the
runs must differ, and the measurement's SUM / MAX reductions must combine them.

One population sharded over ranks: every rank keeps only the rows of the chains it owns
(the ownership rule the device applies) and ``assemble_stage`` must rebuild the whole
stage exactly, with the work counters summed."""
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


def _shard_worker(rank, world, port, outdir):
    from types import SimpleNamespace

    from oracle import tmcmc as tm

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = np.full(3, -8.0), np.full(3, 8.0)
    th = synthetic.prior_samples(5, lo, hi, 512)
    ll = _loglik(th)
    u_res, u_acc, z = synthetic.stage_randoms(5, 0, 512, 3)
    a = tm.analyze(th, ll, 0.0)
    idx = tm.resample(a["w"], u_res)
    m = tm.metropolis(th, ll, idx, a["chol"], a["q_next"], z, u_acc, lo, hi, _loglik)
    counts = np.bincount(idx, minlength=512)
    owner = ranks.chain_owner(counts, world)
    rows = np.concatenate([[owner[k]] * int(counts[k]) for k in range(512) if counts[k] > 0])
    mine = rows == rank
    # this rank's share of the stage (the device leaves zeros in the other ranks' rows)
    st = SimpleNamespace(theta=torch.tensor(np.where(mine[:, None], m["theta"], 0.0)),
                         loglik=torch.tensor(np.where(mine, m["loglik"], 0.0)), surr_loglik=None,
                         c=SimpleNamespace(n_accept=rank + 1, n_exact=10 * (rank + 1), n_screened=0,
                                           n_exact_path=rank))
    ranks.assemble_stage(tdist, st)
    np.savez(os.path.join(outdir, f"shard{rank}.npz"), theta=st.theta.numpy(), loglik=st.loglik.numpy(),
             ref_theta=m["theta"], ref_loglik=m["loglik"], loads=np.bincount(rows, minlength=world),
             counters=np.array([st.c.n_accept, st.c.n_exact, st.c.n_exact_path]), cmax=counts.max())
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


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_stage_assembles_on_gloo_ranks(world):
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_shard_worker, args=(world, port, d), nprocs=world, join=True)
        res = [np.load(os.path.join(d, f"shard{r}.npz")) for r in range(world)]
    for r in res:
        assert np.array_equal(r["theta"], r["ref_theta"]) and np.array_equal(r["loglik"], r["ref_loglik"])
        assert list(r["counters"]) == [sum(range(1, world + 1)), 10 * sum(range(1, world + 1)),
                                       sum(range(world))]
    loads = res[0]["loads"]
    assert loads.sum() == 512 and np.all(np.abs(loads - 512 / world) <= res[0]["cmax"])


def test_chain_owner_rule():
    counts = [0, 3, 1, 0, 4, 2, 0, 6]  # B = 16
    own = ranks.chain_owner(counts, 2)
    # rows: k=1 [0,3) mid 1.5 -> 0; k=2 [3,4) -> 0; k=4 [4,8) mid 6 -> 0; k=5 [8,10) mid 9 -> 1;
    # k=7 [10,16) -> 1
    assert own == {1: 0, 2: 0, 4: 0, 5: 1, 7: 1}
    assert set(ranks.chain_owner(counts, 1).values()) == {0}
