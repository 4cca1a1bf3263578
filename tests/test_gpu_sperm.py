"""GPU parity of the full sperm model (flagellum + head + neck; Appendix, Table Tab:param)
against the oracle through the C ABI: head-centre velocity observations and mean speed
(FP64 1e-10, FP32 1e-4 relative on per-step velocities, 1e-3 on interval velocities), the
proximal point's trajectory with a head attached, the smallest head and uneven flagella."""
import math
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sperm as sp
from oracle import swimmer as sw

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1910_12007_gb300 as g  # noqa: E402

DEV = torch.device("cuda:0")
# Table Tab:param's flagellum and head stiffnesses on a coarser flagellum (20 points)
FLAG = sw.SwimmerParams(n=20, k_t=1e4, k_c=8.0, omega=4 * math.pi, delta_over_ds=0.045 * 19, amp=0.1,
                        alpha=1.0, dt=5e-6, steps=600, obs_every=60)
BASE = sp.SpermParams(FLAG, n_head=8)
THETAS = [(1.0, math.log10(8.0), 0.1), (4.0, 0.5, 0.15), (0.0, 0.9, 0.07)]


def _cfg(p: sp.SpermParams, b_max, precision, observe=g.OBS_HEAD_VELOCITY, **kw):
    f = p.flag
    c = g.SwimmerConfig(n_max=p.nt, b_max=b_max, length=f.length, mu=f.mu, delta_over_ds=f.delta_over_ds, dt=f.dt,
                        k_t=f.k_t, eta=f.eta, omega=f.omega, steps=f.steps, obs_every=f.obs_every,
                        precision=precision, n_head=p.n_head, k_head_tens=p.k_head_tens, k_head_c=p.k_head_c,
                        k_neck_tens=p.k_neck_tens, k_neck_ang=p.k_neck_ang, obs_kind=observe)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _theta(thetas):
    return torch.tensor(thetas, dtype=torch.float64, device=DEV)


def _oracle(p, thetas, observe="velocity"):
    out = []
    for t in thetas:
        q = p.with_theta(t)
        obs, X, st = sp.run_numpy(q, observe=observe)
        assert st == 0
        out.append((obs, X, sp.mean_speed(sp.initial_shape(q), X, q, q.flag.steps * q.flag.dt)))
    return out


@pytest.fixture(scope="module")
def oracle_velocity():
    return _oracle(BASE, THETAS)


@pytest.mark.parametrize("precision,tol", [(g.FP64, 1e-10), (g.FP32C, 1e-3)])
def test_head_centre_velocity_matches_oracle(oracle_velocity, precision, tol):
    h = g.swimmer_init(_cfg(BASE, 4, precision))
    traj, speed, status = g.forward_batch(h, _theta(THETAS))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for b, (obs, X, spd) in enumerate(oracle_velocity):
        vg = traj[b].cpu().numpy()
        err = np.max(np.linalg.norm(vg - obs, axis=1)) / np.max(np.linalg.norm(obs, axis=1))
        assert err < tol, (b, err)
        assert abs(speed[b].item() - spd) <= tol * max(abs(spd), np.max(np.abs(obs[:, 0])))
    h.close()


def test_fp32_per_step_head_velocity():
    p = replace(BASE, flag=replace(FLAG, steps=150, obs_every=1))
    ref = _oracle(p, THETAS[:2])
    h = g.swimmer_init(_cfg(p, 2, g.FP32C))
    traj, _, status = g.forward_batch(h, _theta(THETAS[:2]))
    torch.cuda.synchronize()
    for b, (obs, _, _) in enumerate(ref):
        err = np.max(np.linalg.norm(traj[b].cpu().numpy() - obs, axis=1)) / np.max(np.linalg.norm(obs, axis=1))
        assert err < 1e-4, (b, err)
    h.close()


@pytest.mark.parametrize("precision,tol", [(g.FP64, 1e-10), (g.FP32C, 1e-3)])
def test_proximal_point_with_head_matches_oracle(precision, tol):
    p = replace(BASE, n_head=4, flag=replace(FLAG, steps=400, obs_every=40))
    ref = _oracle(p, THETAS[:2], observe="point")
    h = g.swimmer_init(_cfg(p, 2, precision, observe=g.OBS_HEAD_POINT))
    traj, _, status = g.forward_batch(h, _theta(THETAS[:2]))
    torch.cuda.synchronize()
    x0 = sp.initial_shape(p)[p.nf - 1]
    for b, (obs, _, _) in enumerate(ref):
        dr = obs - x0
        dg = traj[b].cpu().numpy() - x0
        err = np.max(np.abs(dg - dr)) / np.max(np.abs(dr))
        assert err < tol, (b, err)
    h.close()


def test_uneven_flagella_with_head():
    # fixed ds, flagella of 12 and 20 points with the same head in one launch
    ds = 1.0 / 19
    p20 = BASE
    p12 = replace(BASE, flag=replace(FLAG, n=12, length=11 * ds))
    r20 = _oracle(p20, [THETAS[0]])[0]
    r12 = _oracle(p12, [THETAS[1]])[0]
    h = g.swimmer_init(_cfg(BASE, 2, g.FP64, ds_fixed=ds))
    traj, _, status = g.forward_batch(h, _theta([THETAS[1], THETAS[0]]),
                                      n_pts=torch.tensor([12, 20], dtype=torch.int32, device=DEV))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for b, ref in ((0, r12), (1, r20)):
        obs = ref[0]
        err = np.max(np.linalg.norm(traj[b].cpu().numpy() - obs, axis=1)) / np.max(np.linalg.norm(obs, axis=1))
        assert err < 1e-10, (b, err)
    h.close()


def test_head_model_rejects_bad_configs():
    for kw in ({"n_head": 5}, {"n_head": 2}, {"obs_kind": g.OBS_HEAD_VELOCITY, "n_head": 0}):
        c = _cfg(BASE, 1, g.FP32C)
        for k, v in kw.items():
            setattr(c, k, v)
        with pytest.raises(RuntimeError):
            g.swimmer_init(c)


# two swimmers (Sec. 4.2): distances between the tail tips and between the head centres
PAIR = sp.PairParams(replace(BASE, flag=replace(FLAG, n=12, delta_over_ds=0.045 * 11, steps=400, obs_every=40)),
                     d=0.5)


def _pair_cfg(q: sp.PairParams, b_max, precision, sigma_ratio=0.0):
    c = _cfg(q.one, b_max, precision, observe=g.OBS_PAIR_DISTANCES)
    c.n_max = q.nt
    c.n_swimmers = 2
    c.swimmer_distance = q.d
    c.sigma_ratio = sigma_ratio
    return c


@pytest.fixture(scope="module")
def pair_oracle():
    out = []
    for t in THETAS[:2]:
        q = sp.PairParams(PAIR.one.with_theta(t), PAIR.d)
        obs, X, st = sp.pair_run_numpy(q)
        assert st == 0
        out.append(obs)
    return out


@pytest.mark.parametrize("precision,tol", [(g.FP64, 1e-10), (g.FP32C, 1e-4)])
def test_two_swimmer_distances_match_oracle(pair_oracle, precision, tol):
    h = g.swimmer_init(_pair_cfg(PAIR, 2, precision))
    traj, _, status = g.forward_batch(h, _theta(THETAS[:2]))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for b, obs in enumerate(pair_oracle):
        # distances change by O(1e-2) from d: compare the changes
        dg = traj[b].cpu().numpy() - PAIR.d
        dr = obs - PAIR.d
        err = np.max(np.abs(dg - dr)) / np.max(np.abs(dr))
        assert err < tol, (b, err)
    h.close()


def test_two_sigma_log_likelihood(pair_oracle):
    D = pair_oracle[0] + np.array([0.002, -0.004]) * synthetic_normals(pair_oracle[0].shape)
    st, ratio = 0.003, 2.5
    ref = [sp.log_likelihood_two_sigma(obs, D, st, ratio * st) for obs in pair_oracle]
    h = g.swimmer_init(_pair_cfg(PAIR, 2, g.FP64, sigma_ratio=ratio))
    ll, status = g.loglik_batch(h, _theta(THETAS[:2]), torch.tensor(D, device=DEV), st)
    torch.cuda.synchronize()
    assert np.allclose(ll.cpu().numpy(), ref, rtol=1e-9, atol=1e-6)
    h.close()


def synthetic_normals(shape):
    import synthetic

    return synthetic.normals(77, synthetic.NOISE, 0, int(np.prod(shape))).reshape(shape)
