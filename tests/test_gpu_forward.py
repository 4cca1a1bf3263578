"""GPU parity of the table build (K1) and the fused forward/likelihood kernel (K2)
against the FP64 oracle, through the C ABI (Python binding = argument marshalling).

Tolerances (stated by the method's precision plan): FP64 kernel 1e-10 relative on
trajectories; FP32-compensated kernel 1e-4 relative on velocities and 1e-3 relative on
net displacement; FP64 table 1e-12, FP32 table 2e-6 against the pointwise definition.
"""
import math
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic
from oracle import brinkmanlet as bk
from oracle import swimmer as sw

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1910_12007_gb300 as g  # noqa: E402

DEV = torch.device("cuda:0")


def _cfg(p: sw.SwimmerParams, b_max, precision, **kw):
    c = g.SwimmerConfig(n_max=p.n, b_max=b_max, length=p.length, mu=p.mu, delta_over_ds=p.delta_over_ds,
                        dt=p.dt, k_t=p.k_t, eta=p.eta, omega=p.omega, steps=p.steps,
                        obs_every=p.obs_every, precision=precision)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _theta(ps):
    return torch.tensor([[p.alpha, math.log10(p.k_c), p.amp] for p in ps], dtype=torch.float64, device=DEV)


# ---------------------------------------------------------------------------------
# K1: kernel tables
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("alpha", [0.0, 1e-3, 1.0, 9.5, 50.0])
def test_kernel_table_matches_oracle(alpha):
    delta = 1.5 / 127
    r_max = 1.25
    h = g.swimmer_init(g.SwimmerConfig(n_max=128, b_max=1, steps=1, obs_every=1))
    rng = np.random.default_rng(7)
    r = np.concatenate([[0.0, 1e-7, 0.3 * delta, delta, 4 * delta, 1.2], rng.uniform(0, r_max, 14),
                        rng.uniform(0, 5 * delta, 10)])
    rt = torch.tensor(r, dtype=torch.float64, device=DEV)
    g1_64, g2_64 = g.swimmer_kernel_eval(h, alpha, delta, r_max, rt, g.FP64)
    g1_32, g2_32 = g.swimmer_kernel_eval(h, alpha, delta, r_max, rt, g.FP32C)
    torch.cuda.synchronize()
    ref = np.array([bk.kernel_g(x, alpha, delta) for x in r])
    s1 = np.maximum(np.abs(ref[:, 0]), 0.05)  # g1 crosses zero at large alpha r
    e64_1 = np.max(np.abs(g1_64.cpu().numpy() - ref[:, 0]) / s1)
    e64_2 = np.max(np.abs(g2_64.cpu().numpy() - ref[:, 1]) / np.abs(ref[:, 1]))
    e32_1 = np.max(np.abs(g1_32.cpu().numpy() - ref[:, 0]) / s1)
    e32_2 = np.max(np.abs(g2_32.cpu().numpy() - ref[:, 1]) / np.abs(ref[:, 1]))
    assert e64_1 < 1e-12 and e64_2 < 1e-12, (e64_1, e64_2)
    assert e32_1 < 2e-6 and e32_2 < 2e-6, (e32_1, e32_2)
    h.close()


def test_kernel_eval_rejects_bad_arguments():
    h = g.swimmer_init(g.SwimmerConfig(n_max=16, b_max=1, steps=1, obs_every=1))
    rt = torch.zeros(3, dtype=torch.float64, device=DEV)
    with pytest.raises(RuntimeError):
        g.swimmer_kernel_eval(h, -1.0, 0.01, 1.0, rt)
    with pytest.raises(RuntimeError):
        g.swimmer_kernel_eval(h, 1.0, 0.0, 1.0, rt)
    h.close()


# ---------------------------------------------------------------------------------
# K2: forward model and likelihood
# ---------------------------------------------------------------------------------
SMALL = sw.SwimmerParams(n=24, dt=2e-5, steps=1500, obs_every=50, alpha=1.0, amp=0.12, k_c=1.0)
THETAS = [(1.0, 0.0, 0.12), (0.0, -0.5, 0.08), (7.3, 0.3, 0.18)]


def _oracle_batch(base, thetas, steps=None):
    ps = [base.with_theta(t) for t in thetas]
    obs, Xf, xc, st = sw.run_c_batch(ps, steps=steps)
    return ps, obs, xc, st


@pytest.fixture(scope="module")
def small_oracle():
    return _oracle_batch(SMALL, THETAS)


def test_forward_fp64_matches_oracle(small_oracle):
    ps, obs, xc, st = small_oracle
    h = g.swimmer_init(_cfg(SMALL, 8, g.FP64))
    traj, speed, status = g.forward_batch(h, _theta(ps))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0) and np.all(st == 0)
    x0 = np.array([SMALL.length, 0.0])
    disp_ref = obs - x0
    disp = traj.cpu().numpy() - x0
    err = np.max(np.abs(disp - disp_ref)) / np.max(np.abs(disp_ref))
    assert err < 1e-10, err
    sp_ref = (xc[:, 1] - xc[:, 0]) / (SMALL.steps * SMALL.dt)
    assert np.max(np.abs(speed.cpu().numpy() - sp_ref) / np.abs(sp_ref)) < 1e-9
    h.close()


def test_forward_fp32_matches_oracle(small_oracle):
    ps, obs, xc, st = small_oracle
    h = g.swimmer_init(_cfg(SMALL, 8, g.FP32C))
    traj, speed, status = g.forward_batch(h, _theta(ps))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    x0 = np.array([SMALL.length, 0.0])
    disp_ref = obs - x0
    disp = traj.cpu().numpy() - x0
    for b in range(len(ps)):
        err = np.max(np.linalg.norm(disp[b] - disp_ref[b], axis=1)) / np.max(np.linalg.norm(disp_ref[b], axis=1))
        assert err < 1e-3, (b, err)
    h.close()


def test_fp32_velocities_match_oracle():
    # head velocity at every step (obs_every = 1): 1e-4 relative to the largest velocity
    p = replace(SMALL, steps=300, obs_every=1)
    ps, obs, xc, st = _oracle_batch(p, THETAS)
    h = g.swimmer_init(_cfg(p, 4, g.FP32C))
    traj, _, status = g.forward_batch(h, _theta(ps))
    torch.cuda.synchronize()
    x0 = np.array([[p.length, 0.0]])
    for b in range(len(ps)):
        vr = np.diff(np.concatenate([x0, obs[b]]), axis=0) / p.dt
        vg = np.diff(np.concatenate([x0, traj[b].cpu().numpy()]), axis=0) / p.dt
        err = np.max(np.linalg.norm(vg - vr, axis=1)) / np.max(np.linalg.norm(vr, axis=1))
        assert err < 1e-4, (b, err)
    h.close()


def test_loglik_matches_oracle(small_oracle):
    ps, obs, xc, st = small_oracle
    D = obs[0] + 0.002 * synthetic.normals(3, synthetic.NOISE, 0, obs[0].size).reshape(obs[0].shape)
    sigma = 0.002
    ref = np.array([sw.log_likelihood(obs[b], D, sigma) for b in range(len(ps))])
    # FP64: to rounding, on the scale of the log-likelihoods' spread.  FP32: a head trajectory
    # that deviates from the FP64 one by at most d per observation changes
    # l = -sum r^2 / (2 sigma^2) by at most (sum |r| d + n d^2 / 2) / sigma^2 (r the FP64
    # residuals, n their count); d = 1e-4 of the head's largest displacement, forty times the
    # FP32 kernel's largest measured trajectory error (2.3e-6 of the displacement)
    x0 = np.array([SMALL.length, 0.0])
    for prec in (g.FP64, g.FP32C):
        h = g.swimmer_init(_cfg(SMALL, 8, prec))
        ll, status = g.loglik_batch(h, _theta(ps), torch.tensor(D, device=DEV), sigma)
        torch.cuda.synchronize()
        ll = ll.cpu().numpy()
        if prec == g.FP64:
            assert np.max(np.abs(ll - ref)) < 1e-9 * max(1.0, np.max(np.abs(ref - ref.max()))), (ll, ref)
        else:
            for b in range(len(ps)):
                d = 1e-4 * np.max(np.linalg.norm(obs[b] - x0, axis=1))
                r = np.abs(D - obs[b])
                bound = (np.sum(r) * d + r.size * d * d / 2) / sigma ** 2
                assert abs(ll[b] - ref[b]) <= bound, (b, ll[b] - ref[b], bound)
        h.close()


def test_ragged_and_edge_cases():
    # n = 3 (minimum), alpha = 0 (Stokes), a bad sample (alpha < 0), uneven n via ds_fixed
    base = replace(SMALL, steps=400, obs_every=40)
    ds = 1.0 / 23
    thetas = [(1.0, 0.0, 0.1), (0.0, 0.0, 0.1), (-1.0, 0.0, 0.1), (2.0, -0.3, 0.15)]
    ns = [24, 7, 24, 3]
    ps = [replace(base.with_theta(t), n=n, length=(n - 1) * ds) for t, n in zip(thetas, ns)]
    ok = [0, 1, 3]
    obs, Xf, xc, st = sw.run_c_batch([ps[i] for i in ok])
    for prec, tol in [(g.FP64, 1e-10), (g.FP32C, 1e-3)]:
        h = g.swimmer_init(_cfg(base, 8, prec, ds_fixed=ds))
        n_pts = torch.tensor(ns, dtype=torch.int32, device=DEV)
        traj, speed, status = g.forward_batch(h, _theta(ps), n_pts=n_pts)
        torch.cuda.synchronize()
        s = status.cpu().numpy()
        assert list(s) == [0, 0, 2, 0]
        assert np.all(np.isnan(traj[2].cpu().numpy()))
        for k, i in enumerate(ok):
            x0 = np.array([ps[i].length, 0.0])
            dr = obs[k] - x0
            dg = traj[i].cpu().numpy() - x0
            scale = max(np.max(np.abs(dr)), 1e-12)
            assert np.max(np.abs(dg - dr)) / scale < tol, (prec, i)
        h.close()


def test_divergence_is_flagged():
    p = replace(SMALL, n=24, dt=4e-4, steps=400, obs_every=40, k_c=5.0)
    _, _, st = sw.run_numpy(p)
    assert st == 1
    for prec in (g.FP64, g.FP32C):
        h = g.swimmer_init(_cfg(p, 2, prec))
        th = _theta([p])
        traj, speed, status = g.forward_batch(h, th)
        ll, st2 = g.loglik_batch(h, th, torch.zeros((p.n_obs, 2), dtype=torch.float64, device=DEV), 0.1)
        torch.cuda.synchronize()
        assert status.item() == 1 and st2.item() == 1
        assert ll.item() == -math.inf
        assert math.isnan(speed.item())
        h.close()


def test_bad_arguments_raise():
    h = g.swimmer_init(_cfg(SMALL, 2, g.FP32C))
    th = _theta([SMALL] * 3)  # B = 3 > b_max = 2
    with pytest.raises(RuntimeError):
        g.forward_batch(h, th)
    with pytest.raises(RuntimeError):
        g.loglik_batch(h, th[:1], torch.zeros((SMALL.n_obs, 2), dtype=torch.float64, device=DEV), -1.0)
    h.close()
    with pytest.raises(RuntimeError):
        g.swimmer_init(g.SwimmerConfig(n_max=2000))


def test_config1_full_size_fp64():
    # the single-forward-run workload at its full size: N = 64, one beat (8e4 steps)
    p = sw.SwimmerParams()
    ps, obs, xc, st = _oracle_batch(p, [(1.0, 0.0, 0.1)])
    assert st[0] == 0
    for prec, tol in [(g.FP64, 1e-10), (g.FP32C, 1e-3)]:
        h = g.swimmer_init(_cfg(p, 1, prec))
        traj, speed, status = g.forward_batch(h, _theta(ps))
        torch.cuda.synchronize()
        x0 = np.array([p.length, 0.0])
        dr = obs[0] - x0
        dg = traj[0].cpu().numpy() - x0
        err = np.max(np.abs(dg - dr)) / np.max(np.abs(dr))
        assert err < tol, (prec, err)
        sp_ref = (xc[0, 1] - xc[0, 0]) / (p.steps * p.dt)
        assert abs(speed.item() - sp_ref) / abs(sp_ref) < (1e-9 if prec == g.FP64 else 1e-3)
        h.close()


WORKLOAD = sw.SwimmerParams(n=128, dt=1e-4 / 64, steps=2000, obs_every=100, k_t=1e3)
PICK = [0, 1, 333, 700, 1023]


@pytest.fixture(scope="module")
def workload_batch():
    rng = np.random.default_rng(11)
    B = 1024
    th = np.column_stack([rng.uniform(0.0, 10.0, B), rng.uniform(-1.0, 0.2, B), rng.uniform(0.05, 0.2, B)])
    return th, _oracle_batch(WORKLOAD, [tuple(th[i]) for i in PICK])


@pytest.mark.parametrize("threads", [128, 256, 512, 128 | g.SHAPE_WIDE, 256 | g.SHAPE_WIDE])
def test_tmcmc_workload_full_batch_sampled(threads, workload_batch):
    # the TMCMC workload's sizes in the launch configurations its autotuner picks: 1024 samples
    # of N = 128 (four blocks of 32: diagonal, circulant and opposite block pairs) in one
    # persistent launch; sampled runs (including the batch's first and last) against the oracle,
    # 2000 of the workload's time steps (every step has the same arithmetic)
    p, pick, B = WORKLOAD, PICK, 1024
    th, (ps, obs, xc, st) = workload_batch
    assert np.all(st == 0)
    h = g.swimmer_init(_cfg(p, B, g.FP32C))
    g.swimmer_tuning(h, g.FP32C, [threads] * 17)
    traj, speed, status = g.forward_batch(h, torch.tensor(th, device=DEV))
    torch.cuda.synchronize()
    traj = traj.cpu().numpy()
    for k, i in enumerate(pick):
        assert status[i].item() == 0
        x0 = np.array([p.length, 0.0])
        dr = obs[k] - x0
        dg = traj[i] - x0
        err = np.max(np.linalg.norm(dg - dr, axis=1)) / np.max(np.linalg.norm(dr, axis=1))
        assert err < 1e-3, (i, err)
    h.close()


def test_tmcmc_workload_velocities_n128():
    # per-step head velocities at N = 128 (1e-4 relative), FP32 kernel with one- and
    # two-target pair units, and the FP64 kernel
    p = sw.SwimmerParams(n=128, dt=1e-4 / 64, steps=200, obs_every=1, k_t=1e3)
    thetas = [(1.0, 0.0, 0.1), (6.5, -0.6, 0.17), (0.0, 0.1, 0.06)]
    ps, obs, xc, st = _oracle_batch(p, thetas)
    x0 = np.array([[p.length, 0.0]])
    for prec, tol, shape in [(g.FP32C, 1e-4, 0), (g.FP32C, 1e-4, 128 | g.SHAPE_WIDE), (g.FP64, 1e-9, 0)]:
        h = g.swimmer_init(_cfg(p, 4, prec))
        if shape:
            g.swimmer_tuning(h, prec, [shape] * 17)
        traj, _, status = g.forward_batch(h, _theta(ps))
        torch.cuda.synchronize()
        for b in range(len(ps)):
            vr = np.diff(np.concatenate([x0, obs[b]]), axis=0) / p.dt
            vg = np.diff(np.concatenate([x0, traj[b].cpu().numpy()]), axis=0) / p.dt
            err = np.max(np.linalg.norm(vg - vr, axis=1)) / np.max(np.linalg.norm(vr, axis=1))
            assert err < tol, (prec, b, err)
        h.close()


# ---------------------------------------------------------------------------------
# full-size workloads: the large sweep (256 x N = 1024, alpha in [0, 50]) and the uneven
# batch (4096 samples, N in {64, 128, 256, 512} at fixed ds) in the launch shapes their
# autotuner chooses from; sampled runs against the oracle, per-step head velocities
# ---------------------------------------------------------------------------------
LARGE = sw.SwimmerParams(n=1024, dt=1e-4 / 2 ** 15, steps=100, obs_every=1, k_t=1e3)
LARGE_PICK = [0, 97, 255]


@pytest.fixture(scope="module")
def large_batch():
    th = synthetic.prior_samples(3000, (0.0, -1.0, 0.05), (50.0, 0.0, 0.2), 256)
    return th, _oracle_batch(LARGE, [tuple(th[i]) for i in LARGE_PICK])


def _velocity_error(traj_b, obs_b, x0, dt):
    vr = np.diff(np.concatenate([x0, obs_b]), axis=0) / dt
    vg = np.diff(np.concatenate([x0, traj_b]), axis=0) / dt
    return np.max(np.linalg.norm(vg - vr, axis=1)) / np.max(np.linalg.norm(vr, axis=1))


@pytest.mark.parametrize("shape", [512 | g.SHAPE_QUAD, 512 | g.SHAPE_WIDE, 512, 256 | g.SHAPE_QUAD, 128])
def test_large_sweep_sampled(shape, large_batch):
    # 512 threads: one CTA per SM, the 128-register instantiation (four-target units run
    # there); 128: the 64-register one
    th, (ps, obs, xc, st) = large_batch
    assert np.all(st == 0)
    p = LARGE
    h = g.swimmer_init(g.SwimmerConfig(n_max=1024, b_max=256, dt=p.dt, steps=p.steps, obs_every=1, k_t=p.k_t,
                                       precision=g.FP32C))
    g.swimmer_tuning(h, g.FP32C, [shape] * 17)
    traj, _, status = g.forward_batch(h, torch.tensor(th, device=DEV))
    torch.cuda.synchronize()
    traj = traj.cpu().numpy()
    x0 = np.array([[p.length, 0.0]])
    for k, i in enumerate(LARGE_PICK):
        assert status[i].item() == 0
        err = _velocity_error(traj[i], obs[k], x0, p.dt)
        assert err < 1e-4, (shape, i, err)
    h.close()


def test_uneven_full_batch_sampled():
    # 4096 samples, fixed ds = 1/255 (L = (N - 1) ds), longest first in one launch, autotuned
    ds, B, steps = 1.0 / 255, 4096, 100
    ns = synthetic.choice_n(2000, [64, 128, 256, 512], B).astype(np.int32)
    th = synthetic.prior_samples(2000, (0.0, -1.0, 0.05), (10.0, 0.0, 0.2), B)
    h = g.swimmer_init(g.SwimmerConfig(n_max=512, b_max=B, ds_fixed=ds, dt=1e-4 / 512, steps=steps, obs_every=1,
                                       precision=g.FP32C))
    tuned = g.swimmer_autotune(h, steps=20)
    traj, _, status = g.forward_batch(h, torch.tensor(th, device=DEV), torch.tensor(ns, device=DEV))
    torch.cuda.synchronize()
    traj = traj.cpu().numpy()
    pick = [int(np.nonzero(ns == n)[0][0]) for n in (64, 128, 256, 512)] + [B - 1]
    base = sw.SwimmerParams(n=512, dt=1e-4 / 512, steps=steps, obs_every=1)
    ps = [replace(base.with_theta(tuple(th[i])), n=int(ns[i]), length=(int(ns[i]) - 1) * ds) for i in pick]
    obs, _, _, st = sw.run_c_batch(ps)
    assert np.all(st == 0)
    for k, i in enumerate(pick):
        assert status[i].item() == 0
        err = _velocity_error(traj[i], obs[k], np.array([[ps[k].length, 0.0]]), base.dt)
        assert err < 1e-4, (i, int(ns[i]), tuned, err)
    h.close()


@pytest.mark.parametrize("shape", [512 | g.SHAPE_QUAD, 256 | g.SHAPE_WIDE])
def test_ragged_sizes_multi_target_units(shape):
    # sizes that are not multiples of 32 (a padded last block) up to the 1024-point maximum,
    # in one launch whose shared memory makes it a 128-register launch; four- and two-target
    # units over 1 .. 32 blocks; every run against the oracle, per-step head velocities
    ds, steps = 1.0 / 255, 60
    ns = np.array([1000, 777, 545, 300, 1024, 33, 65, 129], dtype=np.int32)
    th = synthetic.prior_samples(21, (0.0, -1.0, 0.05), (10.0, 0.0, 0.2), len(ns))
    dt = 1e-4 / 2 ** 12
    h = g.swimmer_init(g.SwimmerConfig(n_max=1024, b_max=len(ns), ds_fixed=ds, dt=dt, steps=steps, obs_every=1,
                                       precision=g.FP32C))
    g.swimmer_tuning(h, g.FP32C, [shape] * 17)
    traj, _, status = g.forward_batch(h, torch.tensor(th, device=DEV), torch.tensor(ns, device=DEV))
    torch.cuda.synchronize()
    traj = traj.cpu().numpy()
    base = sw.SwimmerParams(n=1024, dt=dt, steps=steps, obs_every=1)
    ps = [replace(base.with_theta(tuple(t)), n=int(n), length=(int(n) - 1) * ds) for t, n in zip(th, ns)]
    obs, _, _, st = sw.run_c_batch(ps)
    assert np.all(st == 0) and np.all(status.cpu().numpy() == 0)
    for b in range(len(ns)):
        err = _velocity_error(traj[b], obs[b], np.array([[ps[b].length, 0.0]]), dt)
        assert err < 1e-4, (shape, int(ns[b]), err)
    h.close()
