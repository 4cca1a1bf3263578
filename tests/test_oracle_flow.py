"""Pins of the oracle's flow and pressure at target points (Eqs. BrP, BrV): the pressure kernel against quadrature of the blob, its singular far field, the
velocity field's zero divergence (incompressible Brinkman flow), and agreement with the pair
sum at the swimmer's own points."""
import math

import numpy as np
from scipy import integrate

from oracle import brinkmanlet as bk
from oracle import swimmer as sw


def test_pressure_kernel_is_the_blob_moment_over_r_squared():
    delta = 0.03
    for r in (0.0, 1e-3, 0.02, 0.1, 1.3):
        if r == 0.0:
            want = 3.0 / (4.0 * math.pi * delta ** 2)  # limit of M0(r)/r^2: phi(0)/2
        else:
            m0, _ = integrate.quad(lambda s: s * bk.blob(s, delta), 0.0, r, epsabs=0, epsrel=1e-13)
            want = m0 / (r * r)
        assert abs(sw.pressure_kernel(r, delta) - want) <= 1e-12 * want


def test_single_force_pressure_far_field():
    # one point force: far from the blob p = (F . d) / (2 pi r^2), the singular solution
    delta = 0.01
    X = np.zeros((1, 2))
    F = np.array([[0.3, -0.7]])
    tab = sw.KernelTable(1.0, delta, 5.0)
    grid = np.array([[2.0, 1.0], [-1.5, 3.0], [0.5, -4.0]])
    _, p = sw.flow_field(X, F, grid, tab, delta)
    want = (grid @ F[0]) / (2 * math.pi * np.sum(grid ** 2, axis=1))
    assert np.allclose(p, want, rtol=1e-9)


def _swimmer_state(alpha=1.5):
    p = sw.SwimmerParams(n=16, alpha=alpha, amp=0.15, steps=1)
    X = sw.initial_shape(p) + np.array([[0.0, 0.02 * math.sin(7 * k / 16)] for k in range(16)])
    F = sw.forces(X, p, 0.13)
    return p, X, F


def test_flow_is_divergence_free():
    p, X, F = _swimmer_state()
    tab = sw.KernelTable(p.alpha, p.delta, 3.0)
    h = 1e-4
    pts = np.array([[0.3, 0.2], [0.8, -0.15], [1.4, 0.05], [-0.2, 0.4]])
    for x in pts:
        g = np.array([x + [h, 0], x - [h, 0], x + [0, h], x - [0, h]])
        v, _ = sw.flow_field(X, F, g, tab, p.delta)
        div = (v[0, 0] - v[1, 0]) / (2 * h) + (v[2, 1] - v[3, 1]) / (2 * h)
        grad = np.max(np.abs([(v[0] - v[1]) / (2 * h), (v[2] - v[3]) / (2 * h)]))
        assert abs(div) < 1e-5 * grad, (x, div, grad)


def test_flow_at_the_swimmer_points_is_the_pair_sum():
    p, X, F = _swimmer_state()
    tab = sw.KernelTable(p.alpha, p.delta, 3.0)
    v, _ = sw.flow_field(X, F, X, tab, p.delta)
    assert np.allclose(v, sw.velocity(X, F, tab), rtol=1e-13, atol=1e-13 * np.max(np.abs(v)))
