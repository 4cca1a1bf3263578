"""Uneven-size batches in one persistent launch (longest first), and CUDA-graph replay of
the whole forward path, against eager launches and the oracle."""
import math
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic
from oracle import swimmer as sw

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1910_12007_gb300 as g  # noqa: E402

DEV = torch.device("cuda:0")
DS = 1.0 / 47


def _cfg(b_max, precision, steps=600, obs_every=60, n_max=48):
    # fixed ds: length = (n - 1) ds per sample
    return g.SwimmerConfig(n_max=n_max, b_max=b_max, ds_fixed=DS, dt=2e-5, steps=steps, obs_every=obs_every,
                           precision=precision)


def _batch(B, seed=4):
    ns = synthetic.choice_n(seed, [6, 12, 24, 48], B).astype(np.int32)
    th = synthetic.prior_samples(seed, (0.2, -0.5, 0.05), (8.0, 0.5, 0.15), B)
    return th, ns


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-3)])
def test_uneven_batch_matches_oracle(precision, tol):
    th, ns = _batch(12)
    h = g.swimmer_init(_cfg(16, precision))
    traj, speed, status = g.forward_batch(h, torch.tensor(th, device=DEV), torch.tensor(ns, device=DEV))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    base = sw.SwimmerParams(n=48, dt=2e-5, steps=600, obs_every=60)
    ps = [replace(base.with_theta(t), n=int(n), length=(int(n) - 1) * DS) for t, n in zip(th, ns)]
    obs, _, _, st = sw.run_c_batch(ps)
    for b in range(len(ps)):
        x0 = np.array([ps[b].length, 0.0])
        dr = obs[b] - x0
        dg = traj[b].cpu().numpy() - x0
        assert np.max(np.abs(dg - dr)) / np.max(np.abs(dr)) < tol, (b, ns[b])
    h.close()


def test_uneven_batch_independent_of_grouping():
    # the longest-first order and the per-sample launch shape do not change any sample's result
    th, ns = _batch(40, seed=9)
    h = g.swimmer_init(_cfg(64, 1))
    thd = torch.tensor(th, device=DEV)
    nsd = torch.tensor(ns, device=DEV)
    traj, _, _ = g.forward_batch(h, thd, nsd)
    for n in np.unique(ns):
        sel = np.nonzero(ns == n)[0]
        t2, _, _ = g.forward_batch(h, thd[sel].contiguous(), nsd[sel].contiguous())
        assert torch.equal(t2, traj[sel]), n
    h.close()


def test_graph_replay_equals_eager():
    th, ns = _batch(32, seed=5)
    h = g.swimmer_init(_cfg(32, 1))
    thd = torch.tensor(th, device=DEV)
    nsd = torch.tensor(ns, device=DEV)
    graph = g.ForwardGraph(h, thd, nsd, want_traj=True)
    th2 = synthetic.prior_samples(6, (0.2, -0.5, 0.05), (8.0, 0.5, 0.15), 32)
    graph.theta.copy_(torch.tensor(th2, device=DEV))
    traj_g, speed_g, st_g = graph.replay()
    torch.cuda.synchronize()
    traj_e, speed_e, st_e = g.forward_batch(h, torch.tensor(th2, device=DEV), nsd)
    torch.cuda.synchronize()
    assert torch.equal(traj_g, traj_e) and torch.equal(speed_g, speed_e) and torch.equal(st_g, st_e)
    h.close()
