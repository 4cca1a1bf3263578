"""Pins of the oracle's Brinkmanlet kernel functions against what the mathematics fixes.

Each test checks the oracle against something other than itself: the printed blob
normalisation (Sec. 2.1, after Eq. eqnblob), high-precision Bessel functions (mpmath),
the independent Fourier/Hankel form of the kernel, the defining ODE
(Lap - alpha^2) B = G (text after Eq. BrV), the singular Brinkmanlet limit delta -> 0,
the regularized Stokeslet limit alpha -> 0 (Cortez 2001) and the positivity of the
mobility operator.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import brinkmanlet as bk

DELTA = 1.5 / 63


def test_blob_normalisation():
    # int_0^inf r phi dr = 1/(2 pi) (printed after Eq. eqnblob)
    val = integrate.quad(lambda r: r * bk.blob(r, DELTA), 0, np.inf, epsabs=0, epsrel=1e-13)[0]
    assert abs(val * 2 * math.pi - 1.0) < 1e-12
    # closed form M0 against quadrature at finite r, including r << delta
    for r in [1e-4 * DELTA, 0.3 * DELTA, DELTA, 7 * DELTA]:
        q = integrate.quad(lambda s: s * bk.blob(s, DELTA), 0, r, epsabs=0, epsrel=2e-14)[0]
        assert abs(bk.m0(r, DELTA) / q - 1.0) < 1e-13


def test_laplace_green_function():
    # phi = Lap G with G' = M0/r:  (1/r) d/dr (r G') = phi
    for r in [0.2 * DELTA, DELTA, 4 * DELTA]:
        h = 1e-4 * r
        d = ((r + h) * bk.g_laplace_prime(r + h, DELTA) - (r - h) * bk.g_laplace_prime(r - h, DELTA)) / (2 * h)
        assert abs(d / r / bk.blob(r, DELTA) - 1.0) < 1e-7


@pytest.mark.parametrize("x", [1e-7, 1e-3, 0.05, 0.7, 1.5, 2.0, 2.5, 9.0, 40.0])
def test_bessel_pieces_against_mpmath(x):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    X = mp.mpf(x)
    k0 = mp.besselk(0, X)
    k2 = mp.besselk(2, X)
    ref = {
        "two_over_x2_minus_k2": 2 / X ** 2 - k2,
        "k0": k0,
        "inv_x2_minus_w": 1 / X ** 2 - (k0 + k2) / 2,
        "i0_minus_1": mp.besseli(0, X) - 1,
    }
    for name, r in ref.items():
        got = getattr(bk, name)(x)
        assert abs(got - float(r)) <= 2e-14 * abs(float(r)) + 1e-300, (name, got, float(r))


@pytest.mark.parametrize("alpha", [0.05, 1.0, 10.0, 50.0])
@pytest.mark.parametrize("rho", [0.0, 0.4, 1.0, 3.0, 12.0])
def test_kernel_matches_hankel_transform(alpha, rho):
    r = rho * DELTA
    g1, g2 = bk.kernel_g(r, alpha, DELTA)
    h1, h2 = bk.hankel_g(r, alpha, DELTA)
    scale1 = max(abs(h1), 1e-3)  # g1 crosses zero at large alpha: compare on its O(0.1) scale
    assert abs(g1 - h1) < 1e-11 * scale1 + 1e-13
    assert abs(g2 - h2) < 1e-11 * abs(h2)


@pytest.mark.parametrize("alpha", [0.3, 4.0, 30.0])
@pytest.mark.parametrize("rho", [0.5, 2.0, 9.0])
def test_defining_ode_residual(alpha, rho):
    # (Lap - alpha^2) B = G  =>  B''' + B''/r - B'/r^2 - alpha^2 B' = G'
    # with B'' = g1 and B' = r g1 - r^3 g2
    r = rho * DELTA
    h = 1e-3 * DELTA

    def b1(rr):
        g1, g2 = bk.kernel_g(rr, alpha, DELTA)
        return rr * g1 - rr ** 3 * g2

    g = [bk.kernel_g(r + k * h, alpha, DELTA)[0] for k in (-2, -1, 0, 1, 2)]
    b3 = (g[0] - 8 * g[1] + 8 * g[3] - g[4]) / (12 * h)
    lhs = b3 + g[2] / r - b1(r) / r ** 2 - alpha ** 2 * b1(r)
    rhs = bk.g_laplace_prime(r, DELTA)
    assert abs(lhs - rhs) < 2e-7 * abs(rhs)


def test_singular_limit():
    # delta -> 0 at fixed r: regularized -> singular Brinkmanlet; gap shrinks with r/delta
    alpha, r = 2.0, 0.2
    gaps = []
    for dl in [2e-2, 2e-3, 2e-4]:
        g1, g2 = bk.kernel_g(r, alpha, dl)
        s1, s2 = bk.singular_g(r, alpha)
        gaps.append(max(abs(g1 / s1 - 1), abs(g2 / s2 - 1)))
    assert gaps[2] < 1e-5
    assert gaps[0] > gaps[1] > gaps[2]


def test_stokes_limit():
    # alpha -> 0: g2 -> Stokes g2, and g1 -> Stokes g1 up to an alpha-dependent constant
    r = np.array([0.0, 0.3, 1.0, 4.0, 20.0]) * DELTA
    s1, s2 = bk.stokes_g(r, DELTA)
    for alpha, tol in [(1e-3, 2e-4), (1e-5, 3e-8)]:
        g = np.array([bk.kernel_g(x, alpha, DELTA) for x in r])
        assert np.max(np.abs(g[:, 1] / s2 - 1)) < tol
        d = (g[:, 0] - g[0, 0]) - (s1 - s1[0])
        assert np.max(np.abs(d)) < tol * np.max(np.abs(s1 - s1[0]))


def test_mobility_positive_semidefinite():
    # Fourier symbol phi^(k) (I - k k/k^2)/(k^2 + alpha^2) >= 0  =>  PSD mobility matrix
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 6 * DELTA, size=(14, 2))
    for alpha in [0.5, 8.0]:
        d = X[:, None, :] - X[None, :, :]
        r = np.hypot(d[..., 0], d[..., 1])
        G = np.array([[bk.kernel_g(r[i, j], alpha, DELTA) for j in range(14)] for i in range(14)])
        M = np.zeros((14, 2, 14, 2))
        for a in range(2):
            for b in range(2):
                M[:, a, :, b] = -G[..., 0] * (a == b) + G[..., 1] * d[..., a] * d[..., b]
        # velocity = -sum F g1 + ...; the mobility acting on F is -M's sign convention:
        # v = M F with M = -g1 I + g2 d d^T, and the operator (grad grad - I Lap) B is PSD
        ev = np.linalg.eigvalsh(0.5 * (M.reshape(28, 28) + M.reshape(28, 28).T))
        assert ev.min() > -1e-10 * ev.max()


def test_table_matches_pointwise():
    rng = np.random.default_rng(1)
    for alpha in [0.0, 0.7, 25.0]:
        T = bk.KernelTable(alpha, DELTA, 1.2)
        r = np.concatenate([[0.0, 1e-6 * DELTA], rng.uniform(0, 1.2, 12), rng.uniform(0, 3 * DELTA, 6)])
        g1, g2 = T(r)
        for i, x in enumerate(r):
            e1, e2 = bk.kernel_g(x, alpha, DELTA)
            assert abs(g1[i] - e1) < 1e-12 * max(abs(e1), 0.05)
            assert abs(g2[i] - e2) < 1e-12 * abs(e2)
