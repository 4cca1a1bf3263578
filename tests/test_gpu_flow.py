"""GPU parity of the final state and of the flow and pressure at target points (Eqs. BrP,
BrV) against the oracle through the C ABI: final positions and the
forces there (FP64 1e-10, FP32 1e-3 on displacement), the flow field from a GPU final state
(FP64 table against the oracle's, 1e-9), and the flow of the sperm model's final state."""
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
P = sw.SwimmerParams(n=24, dt=2e-5, steps=500, obs_every=50, alpha=1.5, amp=0.12, k_c=1.0)
THETAS = [(1.5, 0.0, 0.12), (0.0, -0.4, 0.09)]


def _cfg(p, b_max, precision):
    return g.SwimmerConfig(n_max=p.n, b_max=b_max, length=p.length, mu=p.mu, delta_over_ds=p.delta_over_ds,
                           dt=p.dt, k_t=p.k_t, eta=p.eta, omega=p.omega, steps=p.steps, obs_every=p.obs_every,
                           precision=precision)


@pytest.mark.parametrize("precision,tol", [(g.FP64, 1e-10), (g.FP32C, 1e-3)])
def test_final_state_matches_oracle(precision, tol):
    h = g.swimmer_init(_cfg(P, 2, precision))
    _, _, status, state = g.forward_batch_state(h, torch.tensor(THETAS, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    state = state.cpu().numpy()
    for b, t in enumerate(THETAS):
        q = P.with_theta(t)
        _, X, st = sw.run_numpy(q)
        assert st == 0
        X0 = sw.initial_shape(q)
        err = np.max(np.abs((state[b, :, :2] - X0) - (X - X0))) / np.max(np.abs(X - X0))
        assert err < tol, (b, err)
        if precision == g.FP64:
            F = sw.forces(X, q, q.steps * q.dt)
            assert np.max(np.abs(state[b, :, 2:] - F)) <= 1e-8 * np.max(np.abs(F))
    h.close()


def test_flow_field_matches_oracle():
    h = g.swimmer_init(_cfg(P, 1, g.FP64))
    _, _, status, state = g.forward_batch_state(h, torch.tensor(THETAS[:1], dtype=torch.float64, device=DEV))
    q = P.with_theta(THETAS[0])
    xs = np.linspace(-0.5, 1.5, 9)
    ys = np.linspace(-0.6, 0.6, 7)
    grid = np.array([[x, y] for x in xs for y in ys])
    st0 = state[0].contiguous()
    vel, pres = g.swimmer_flow_field(h, q.alpha, q.delta, 3.0, st0, torch.tensor(grid, device=DEV))
    torch.cuda.synchronize()
    S = st0.cpu().numpy()
    tab = sw.KernelTable(q.alpha, q.delta, 3.0)
    v_ref, p_ref = sw.flow_field(S[:, :2], S[:, 2:], grid, tab, q.delta, q.mu)
    assert np.max(np.abs(vel.cpu().numpy() - v_ref)) <= 1e-9 * np.max(np.abs(v_ref))
    assert np.max(np.abs(pres.cpu().numpy() - p_ref)) <= 1e-9 * np.max(np.abs(p_ref))
    # on the swimmer's own points the flow is the pair-sum velocity
    vpts, _ = g.swimmer_flow_field(h, q.alpha, q.delta, 3.0, st0, st0[:, :2].contiguous())
    assert np.allclose(vpts.cpu().numpy(), sw.velocity(S[:, :2], S[:, 2:], tab, q.mu), rtol=1e-9,
                       atol=1e-9 * np.max(np.abs(v_ref)))
    h.close()


def test_sperm_model_final_state_and_flow():
    f = sw.SwimmerParams(n=14, k_t=1e4, k_c=8.0, omega=4 * math.pi, delta_over_ds=0.045 * 13, amp=0.1,
                         alpha=1.0, dt=5e-6, steps=200, obs_every=50)
    q = sp.SpermParams(f, n_head=8)
    cfg = g.SwimmerConfig(n_max=q.nt, b_max=1, length=1.0, delta_over_ds=f.delta_over_ds, dt=f.dt, k_t=f.k_t,
                          omega=f.omega, steps=f.steps, obs_every=f.obs_every, precision=g.FP64, n_head=8,
                          obs_kind=g.OBS_HEAD_VELOCITY)
    h = g.swimmer_init(cfg)
    th = (1.0, math.log10(8.0), 0.1)
    _, _, status, state = g.forward_batch_state(h, torch.tensor([th], dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    _, X, st = sp.run_numpy(q.with_theta(th))
    S = state[0].cpu().numpy()
    X0 = sp.initial_shape(q)
    assert np.max(np.abs((S[:, :2] - X0) - (X - X0))) <= 1e-10 * np.max(np.abs(X - X0))
    F = sp.forces(X, q.with_theta(th), f.steps * f.dt)
    assert np.max(np.abs(S[:, 2:] - F)) <= 1e-8 * np.max(np.abs(F))
    grid = np.array([[0.5, 0.3], [1.3, -0.2], [1.6, 0.1]])
    vel, pres = g.swimmer_flow_field(h, 1.0, f.delta, 3.0, state[0].contiguous(), torch.tensor(grid, device=DEV))
    v_ref, p_ref = sw.flow_field(S[:, :2], S[:, 2:], grid, sw.KernelTable(1.0, f.delta, 3.0), f.delta)
    assert np.max(np.abs(vel.cpu().numpy() - v_ref)) <= 1e-9 * np.max(np.abs(v_ref))
    assert np.max(np.abs(pres.cpu().numpy() - p_ref)) <= 1e-9 * np.max(np.abs(p_ref))
    h.close()
