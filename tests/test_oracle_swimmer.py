"""Pins of the oracle's flagellum model (Appendix Eqs. EFB, curva, EFT; Eq. Fenergy;
Eq. BrV; forward Euler) and likelihood (Eqs. likelihood, fitness)."""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import swimmer as sw

SMALL = sw.SwimmerParams(n=12, dt=2e-5, steps=400, obs_every=40, alpha=1.5)


def _perturbed(p, seed=0, scale=0.01):
    rng = np.random.default_rng(seed)
    return sw.initial_shape(p) + scale * rng.standard_normal((p.n, 2))


def test_forces_are_energy_gradient():
    p = replace(SMALL, n=16, k_c=3.0, amp=0.2)
    X = _perturbed(p)
    F = sw.forces(X, p, 0.37)
    h = 1e-6
    G = np.zeros_like(X)
    for i in range(p.n):
        for c in range(2):
            A = X.copy(); A[i, c] += h
            B = X.copy(); B[i, c] -= h
            G[i, c] = -(sw.energy(A, p, 0.37) - sw.energy(B, p, 0.37)) / (2 * h)
    assert np.max(np.abs(F - G)) < 1e-8 * np.max(np.abs(F))


def test_zero_net_force_and_torque():
    # translation and rotation invariance of the energy (force- and torque-free swimmer)
    p = replace(SMALL, n=20, amp=0.15)
    X = _perturbed(p, 2, 0.02)
    F = sw.forces(X, p, 0.11)
    scale = np.max(np.abs(F)) * p.n
    assert np.max(np.abs(F.sum(0))) < 1e-13 * scale
    torque = np.sum(X[:, 0] * F[:, 1] - X[:, 1] * F[:, 0])
    assert abs(torque) < 1e-13 * scale


def test_preferred_curvature_is_second_derivative():
    p = replace(SMALL, n=30, length=1.3)
    t = 0.21
    s = np.arange(1, p.n - 1) * p.ds
    h = 1e-4
    yhat = lambda ss: p.amp * (1 - ss / p.length) * np.sin(p.eta * ss - p.omega * t)
    fd = (yhat(s + h) - 2 * yhat(s) + yhat(s - h)) / h ** 2
    assert np.max(np.abs(sw.preferred_curvature(p, t) - fd)) < 1e-6 * np.max(np.abs(fd))


def test_straight_filament_stays_at_rest():
    p = replace(SMALL, amp=0.0, steps=300)
    obs, X, st = sw.run_numpy(p)
    assert st == 0
    # no transverse force can arise: y stays exactly zero; x moves only by the rounding
    # of the rest lengths k*ds (relative 1e-16 tension residuals)
    assert np.all(X[:, 1] == 0.0)
    assert np.max(np.abs(X - sw.initial_shape(p))) < 1e-14


def test_mirror_symmetry():
    # y -> -y with a -> -a maps a trajectory onto its mirror image
    p = replace(SMALL, amp=0.1)
    q = replace(SMALL, amp=-0.1)
    T = sw.kernel_table(p)
    o1, X1, _ = sw.run_numpy(p, T)
    o2, X2, _ = sw.run_numpy(q, T)
    assert np.max(np.abs(X1[:, 0] - X2[:, 0])) < 1e-13
    assert np.max(np.abs(X1[:, 1] + X2[:, 1])) < 1e-13


def test_first_order_convergence_in_dt():
    p = replace(SMALL, n=10, amp=0.15, steps=200, obs_every=200, dt=4e-5)
    T = sw.kernel_table(p)
    ends = []
    for k in (1, 2, 4):
        q = replace(p, dt=p.dt / k, steps=p.steps * k, obs_every=p.obs_every * k)
        ends.append(sw.run_c_batch([q], [T])[0][0, -1])
    e1 = np.linalg.norm(ends[0] - ends[1])
    e2 = np.linalg.norm(ends[1] - ends[2])
    assert 1.6 < e1 / e2 < 2.4


def test_c_loop_matches_numpy_loop():
    p = replace(SMALL, amp=0.12, k_c=2.0)
    T = sw.kernel_table(p)
    o1, X1, s1 = sw.run_numpy(p, T)
    o2, X2, xc, s2 = sw.run_c_batch([p], [T])
    assert s1 == 0 and s2[0] == 0
    assert np.max(np.abs(X1 - X2[0])) < 1e-13
    assert np.max(np.abs(o1 - o2[0])) < 1e-13


def test_euler_instability_is_flagged():
    # dt beyond the linear stability bound of forward Euler: the run reports divergence
    p = replace(SMALL, n=24, dt=4e-4, steps=400, k_c=5.0)
    lam = sw.euler_lambda_max(p)
    assert lam * p.dt > 2.0
    _, _, st = sw.run_numpy(p)
    assert st == 1


def test_log_likelihood_hand_computed():
    g = np.array([[1.0, 2.0], [0.5, -1.0], [0.0, 0.25]])
    D = g + np.array([[0.1, -0.2], [0.0, 0.3], [-0.1, 0.0]])
    sigma = 0.2
    J = (0.01 + 0.04 + 0.0 + 0.09 + 0.01 + 0.0) / 0.04
    expect = -0.5 * 6 * math.log(2 * math.pi * 0.04) - 0.5 * J
    assert abs(sw.log_likelihood(g, D, sigma) - expect) < 1e-12
    assert sw.noise_sigma(np.array([1.0, -3.0]), 0.05) == pytest.approx(0.1)


@pytest.mark.parametrize("alpha", [0.0, 1.0, 5.0])
def test_energy_decreases_along_the_flow_with_a_static_preferred_shape(alpha):
    """With omega = 0 the preferred curvature does not move, so E(X) (Eqs. EFB, EFT) is a
    fixed function of the positions and dE/dt = grad E . v = -F . M F <= 0: the Brinkmanlet
    mobility of Eq. BrV is positive semi-definite (its Fourier symbol is the blob's positive
    transform times the Brinkman propagator).  Forward Euler at a step well inside its
    stability bound keeps the decrease step by step.  A flipped velocity (v = -M F) would
    raise the energy at every step."""
    p = sw.SwimmerParams(n=24, dt=5e-5, omega=0.0, amp=0.1, alpha=alpha, k_c=1.0)
    table = sw.kernel_table(p)
    X = sw.initial_shape(p)
    E = [sw.energy(X, p, 0.0)]
    for _ in range(150):
        F = sw.forces(X, p, 0.0)
        X = X + p.dt * sw.velocity(X, F, table, p.mu)
        E.append(sw.energy(X, p, 0.0))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * E[0])
    assert E[-1] < 0.5 * E[0]  # the filament relaxes toward its preferred shape
    # and the same run through the oracle's own time loop ends in the same state
    _, X_loop, status = sw.run_numpy(replace(p, steps=150, obs_every=150), table)
    assert status == 0 and np.allclose(X_loop, X, rtol=0, atol=1e-14)
