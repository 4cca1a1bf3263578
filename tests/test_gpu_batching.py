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


@pytest.mark.parametrize("precision,tol,shape", [(0, 1e-10, 0), (1, 1e-3, 0), (1, 1e-3, 128 | g.SHAPE_WIDE)])
def test_uneven_batch_matches_oracle(precision, tol, shape):
    # N in {6, 12, 24, 48}: one and two blocks of 32 (a lone off-diagonal block pair)
    th, ns = _batch(12)
    h = g.swimmer_init(_cfg(16, precision))
    if shape:
        g.swimmer_tuning(h, precision, [shape] * 17)
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


def test_uniform_batch_independent_of_processing_order():
    # batches of one size are processed in ascending K_C (the runs likely to stop early last);
    # a sample's result must not depend on that order or on which CTA takes it
    B = 64
    th = synthetic.prior_samples(12, (0.2, -1.0, 0.05), (8.0, 1.0, 0.15), B)
    h = g.swimmer_init(_cfg(B, 1))
    thd = torch.tensor(th, device=DEV)
    traj, speed, st = g.forward_batch(h, thd)
    perm = torch.tensor(np.random.default_rng(3).permutation(B), device=DEV)
    traj_p, speed_p, st_p = g.forward_batch(h, thd[perm].contiguous())
    torch.cuda.synchronize()
    same = lambda a, b: torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))  # noqa: E731
    assert same(traj_p, traj[perm]) and torch.equal(st_p, st[perm]) and same(speed_p, speed[perm])
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


def test_launch_shapes_agree_and_tuning_table_round_trips():
    # N up to 96 points: 3 blocks of 32, so 128..512 threads give 4, 8 and 9 pair warps
    cfg = replace(_cfg(64, g.FP32C, steps=300, obs_every=30, n_max=96))
    h = g.swimmer_init(cfg)
    th = torch.tensor(synthetic.prior_samples(9, (0.2, -0.5, 0.05), (8.0, 0.5, 0.15), 40), device=DEV)
    ns = torch.tensor(synthetic.choice_n(9, [40, 70, 96], 40).astype(np.int32), device=DEV)
    outs = {}
    W, Q = g.SHAPE_WIDE, g.SHAPE_QUAD
    # (at N <= 96 every launch keeps the 64-register kernel, so QUAD runs two-target units)
    shapes = (128, 256, 512, 128 | W, 256 | W, 512 | W, 128 | Q)
    for T in shapes:
        g.swimmer_tuning(h, g.FP32C, [T] * 17)
        assert g.swimmer_tuning(h, g.FP32C) == [T] * 17
        traj, speed, st = g.forward_batch(h, th, ns)
        outs[T] = (traj.cpu().numpy(), st.cpu().numpy())
    ref_traj, ref_st = outs[128]
    assert np.all(ref_st == 0)
    scale = np.max(np.abs(ref_traj))
    for T in shapes[1:]:
        # only the grouping of the FP32 partial sums changes with the number of pair warps
        # and with the grouping of block pairs into units
        assert np.array_equal(outs[T][1], ref_st)
        assert np.max(np.abs(outs[T][0] - ref_traj)) <= 1e-5 * scale
    with pytest.raises(RuntimeError):
        g.swimmer_tuning(h, g.FP32C, [96] * 17)  # not a power of two
    with pytest.raises(RuntimeError):
        g.swimmer_tuning(h, g.FP32C, [128 | 0x40000] * 17)  # unknown flag
    with pytest.raises(RuntimeError):
        g.swimmer_tuning(h, g.FP32C, [128 | W | Q] * 17)  # one flag at most
    h64 = g.swimmer_init(replace(cfg, precision=g.FP64))
    with pytest.raises(RuntimeError):
        g.swimmer_tuning(h64, g.FP64, [128 | W] * 17)  # two-target units are FP32 only
    h64.close()
    tuned = g.swimmer_autotune(h, steps=20)
    assert set(tuned) and all(v & ~(W | Q) in (128, 256, 512, 1024) for v in tuned.values())
    table = g.swimmer_tuning(h, g.FP32C)
    assert table[0] == tuned[1]
    h.close()
