"""Pins of the oracle's full sperm model (flagellum + head + neck; Appendix, Table Tab:param)
against the mathematics: exact gradients, rigid-motion invariance, the rest state of the
springs and the neck angle, the closed-form discrete curvature of a regular polygon, the
flagellum-only model when the head terms are off, first-order convergence in dt."""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import sperm as sp
from oracle import swimmer as sw

FLAG = sw.SwimmerParams(n=20, k_t=1e4, k_c=8.0, omega=4 * math.pi, delta_over_ds=0.045 * 19, amp=0.1,
                        alpha=1.0, dt=1e-5, steps=3, obs_every=1)
P = sp.SpermParams(FLAG, n_head=12)


def _fd(X, p, t, h=1e-6):
    G = np.zeros_like(X)
    for i in range(X.shape[0]):
        for c in range(2):
            a = X.copy()
            a[i, c] += h
            b = X.copy()
            b[i, c] -= h
            G[i, c] = -(sp.energy(a, p, t) - sp.energy(b, p, t)) / (2 * h)
    return G


def test_forces_are_the_exact_energy_gradient():
    X = sp.initial_shape(P) + 2e-3 * np.random.default_rng(1).standard_normal((P.nt, 2))
    F = sp.forces(X, P, 0.37)
    G = _fd(X, P, 0.37)
    assert np.max(np.abs(F - G)) <= 1e-7 * np.max(np.abs(G))


def test_zero_net_force_and_torque():
    X = sp.initial_shape(P) + 5e-3 * np.random.default_rng(2).standard_normal((P.nt, 2))
    F = sp.forces(X, P, 1.1)
    scale = np.max(np.abs(F))
    assert np.all(np.abs(F.sum(0)) < 1e-12 * scale * P.nt)
    assert abs(np.sum(X[:, 0] * F[:, 1] - X[:, 1] * F[:, 0])) < 1e-12 * scale * P.nt


def test_springs_and_neck_angle_rest_initially():
    X = sp.initial_shape(P)
    for i, j, k, l0 in sp.springs(P):
        assert abs(np.hypot(*(X[j] - X[i])) - l0) < 1e-15
    f, hp, hplus, hminus = sp.angle_points(P)
    assert abs((X[hp] - X[f]) @ (X[hplus] - X[hminus])) < 1e-15
    # H(pi) faces the flagellum's proximal end at distance dN on its line
    assert np.allclose(X[hp] - X[f], [P.gap, 0.0], atol=1e-15)
    assert len(sp.springs(P)) == P.n_head + P.n_head // 2 + 5


def test_regular_polygon_curvature_closed_form():
    H = sp.initial_shape(P)[P.nf:]
    kap = sp.head_curvature(H, P.ds_head)
    dth = 2 * math.pi / P.n_head
    assert np.allclose(kap, 2.0 / (P.hr * (1.0 + math.cos(dth))), rtol=1e-12)
    # the curvature does not depend on the parameter spacing of the differences
    assert np.allclose(sp.head_curvature(H, 3.7 * P.ds_head), kap, rtol=1e-12)


def test_flagellum_model_when_head_terms_are_off():
    q = replace(P, k_head_tens=0.0, k_head_c=0.0, k_neck_tens=0.0, k_neck_ang=0.0)
    X = sp.initial_shape(q) + 1e-3 * np.random.default_rng(3).standard_normal((q.nt, 2))
    F = sp.forces(X, q, 0.2)
    assert np.array_equal(F[:q.nf], sw.forces(X[:q.nf], q.flag, 0.2))
    assert not F[q.nf:].any()


def test_first_order_in_dt():
    base = sp.SpermParams(replace(FLAG, n=10, delta_over_ds=2.0, dt=2e-5, steps=40, obs_every=40), n_head=8)
    tab = sp.kernel_table(base)
    ends = []
    for r in (1, 2, 4, 8):
        q = replace(base, flag=replace(base.flag, dt=base.flag.dt / r, steps=base.flag.steps * r,
                                       obs_every=base.flag.obs_every * r))
        _, X, st = sp.run_numpy(q, tab)
        assert st == 0
        ends.append(X)
    e = [np.max(np.abs(ends[i] - ends[3])) for i in range(3)]
    # first order: the error against the dt/8 run is C (h - h/8), so the ratios are
    # (1 - 1/8)/(1/2 - 1/8) = 7/3 and (1/2 - 1/8)/(1/4 - 1/8) = 3
    assert abs(e[0] / e[1] - 7.0 / 3.0) < 0.15
    assert abs(e[1] / e[2] - 3.0) < 0.2


# two swimmers (Sec. 4.2)
PAIR = sp.PairParams(replace(P, flag=replace(FLAG, n=12, delta_over_ds=1.5)), d=0.5)


def test_pair_forces_are_the_exact_energy_gradient_and_separate():
    X = sp.pair_initial_shape(PAIR) + 2e-3 * np.random.default_rng(4).standard_normal((PAIR.nt, 2))
    F = sp.pair_forces(X, PAIR, 0.21)
    G = np.zeros_like(X)
    h = 1e-6
    for i in range(X.shape[0]):
        for c in range(2):
            a = X.copy()
            a[i, c] += h
            b = X.copy()
            b[i, c] -= h
            G[i, c] = -(sp.pair_energy(a, PAIR, 0.21) - sp.pair_energy(b, PAIR, 0.21)) / (2 * h)
    assert np.max(np.abs(F - G)) <= 1e-7 * np.max(np.abs(G))
    # each swimmer's forces are its own: zero net force and torque per swimmer
    n = PAIR.one.nt
    for Fs, Xs in ((F[:n], X[:n]), (F[n:], X[n:])):
        assert np.all(np.abs(Fs.sum(0)) < 1e-9 * np.max(np.abs(Fs)) * n)


def test_pair_initial_distances_and_far_field_decay():
    X = sp.pair_initial_shape(PAIR)
    assert np.allclose(sp.pair_distances(X, PAIR), [PAIR.d, PAIR.d], atol=1e-15)
    # each swimmer is force-free, so in a Brinkman fluid the other's influence is the
    # potential-flow dipole far field, ~ d^-3: doubling the separation divides the deviation
    # from a lone swimmer by about 8
    one = replace(PAIR.one, flag=replace(PAIR.one.flag, alpha=2.0, steps=60, obs_every=60))
    dev = []
    for d in (12.0, 24.0):
        far = sp.PairParams(one, d=d)
        _, Xp, st = sp.pair_run_numpy(far)
        _, X1, st1 = sp.run_numpy(one, table=sp.pair_kernel_table(far))
        assert st == 0 and st1 == 0
        n = one.nt
        disp1 = X1 - sp.initial_shape(one)
        dev.append(np.max(np.abs((Xp[:n] - sp.initial_shape(one)) - disp1)) / np.max(np.abs(disp1)))
        # the second swimmer mirrors the first's motion (same start, displaced by d)
        assert np.max(np.abs((Xp[n:] - [0.0, d]) - Xp[:n])) < 10 * dev[-1] * np.max(np.abs(disp1))
    assert dev[1] < 1e-5
    assert 6.5 < dev[0] / dev[1] < 9.5


def test_two_sigma_likelihood_by_hand():
    g = np.array([[1.0, 2.0], [1.5, 2.5]])
    D = np.array([[1.1, 1.8], [1.4, 2.9]])
    st, sh = 0.2, 0.5
    want = (-2 * 0.5 * (math.log(2 * math.pi * 0.04) + math.log(2 * math.pi * 0.25))
            - 0.5 * (0.1 ** 2 + 0.1 ** 2) / 0.04 - 0.5 * (0.2 ** 2 + 0.4 ** 2) / 0.25)
    assert sp.log_likelihood_two_sigma(g, D, st, sh) == pytest.approx(want, rel=1e-14)
    # equal noise levels reduce to the one-sigma likelihood
    assert sp.log_likelihood_two_sigma(g, D, 0.3, 0.3) == pytest.approx(sw.log_likelihood(g, D, 0.3), rel=1e-14)
