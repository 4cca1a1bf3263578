"""Regularized Brinkmanlet kernel functions, FP64 (oracle; test infrastructure only).

What the paper defines (Sec. 2.1)
---------------------------------
* Blob, Eq. (eqnblob): phi_d(r) = 3 d^3 / (2 pi (r^2 + d^2)^(5/2)), with
  int_0^inf r phi dr = 1/(2 pi).
* Velocity, Eq. (BrV): v(x) = sum_i [ -F_i B''(r) + (F_i . d) d (r B'' - B')/r^3 ],
  d = x - X_i, r = |d|, where phi = Lap G and (Lap - alpha^2) B = G (text after Eq. BrV).

The paper defers the closed form of B to other work.  This module evaluates it from the
definition: with G_B the decaying solution of (Lap - alpha^2) G_B = phi, the function
B = (G_B - G)/alpha^2 satisfies (Lap - alpha^2) B = G.  The radial Green's function of
(Lap - alpha^2) in 2D is -K0(alpha|x|)/(2 pi); averaging it over circles (Graf's addition
theorem) gives

    G_B(r) = -K0(a r) int_0^r I0(a s) phi s ds - I0(a r) int_r^inf K0(a s) phi s ds.

Writing M0(r) = int_0^r phi s ds (closed form), A1(r) = int_0^r (I0(a s) - 1) phi s ds,
C(r) = int_r^inf K0(a s) phi s ds and x = a r, the two velocity functions are

    g1(r) = B''(r)             = [1/x^2 - W(x)] M0 - W(x) A1 - (I0(x) + I2(x)) C / 2
    g2(r) = (r B'' - B')/r^3   = [(2/x^2 - K2(x)) M0 - K2(x) A1 - I2(x) C] / r^2

with W = (K0 + K2)/2.  Each line follows from B' = (G_B' - G')/a^2 and
B'' = G_B - B'/r by the Bessel recurrences K2 = K0 + 2 K1/x and I0 - I2 = 2 I1/x; the
bracketed combinations are evaluated from their power series for x <= 2 so that no
catastrophic cancellation occurs as a r -> 0.  At r = 0: g1(0) = -C(0)/2 and
g2(0) = (phi(0) - a^2 C(0))/8.

alpha = 0 is the regularized Stokeslet, whose closed form (Cortez 2001, the same blob) is
used directly:  g1 = [ln(R + d) - d (R + 2d)/(R (R + d))]/(4 pi),
g2 = (R + 2d)/(4 pi R (R + d)^2), R = sqrt(r^2 + d^2).  B'' is only defined up to an
additive constant at alpha = 0 (the 2D Stokes paradox); the constant multiplies the net
force, which is zero for a free swimmer.

Pins (tests/test_oracle_brinkmanlet.py): blob normalisation; the series pieces against
scipy/mpmath Bessel functions; g1, g2 against the independent Hankel-transform form
(2D Fourier transform of phi is (1 + k d) e^{-k d}); the ODE residual
(Lap - alpha^2) B = G; the delta -> 0 singular Brinkmanlet; alpha -> 0 Stokes limit;
positive semi-definiteness of the mobility matrix; the interpolation table against
pointwise evaluation.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special

EULER_GAMMA = 0.57721566490153286060651209008240243


# ---------------------------------------------------------------------------------
# blob and Laplace Green's function (Eq. eqnblob)
# ---------------------------------------------------------------------------------
def blob(r, delta):
    """phi_delta(r) = 3 delta^3 / (2 pi (r^2 + delta^2)^{5/2})  (Eq. eqnblob)."""
    r = np.asarray(r, dtype=np.float64)
    return 3.0 * delta ** 3 / (2.0 * np.pi * (r * r + delta * delta) ** 2.5)


def m0(r, delta):
    """M0(r) = int_0^r phi(s) s ds = (1 - delta^3/R^3)/(2 pi), written without cancellation.

    1 - d^3/R^3 = (R - d)(R^2 + R d + d^2)/R^3 and R - d = r^2/(R + d).
    """
    r = np.asarray(r, dtype=np.float64)
    R = np.hypot(r, delta)
    return (r * r / (R + delta)) * (R * R + R * delta + delta * delta) / R ** 3 / (2.0 * np.pi)


def g_laplace_prime(r, delta):
    """G_delta'(r) = M0(r)/r, the radial derivative of the regularized Laplace Green's
    function (phi = Lap G, text after Eq. BrV)."""
    return m0(r, delta) / r


# ---------------------------------------------------------------------------------
# Bessel combinations (A&S 9.6.11 / 9.6.13 series for small argument)
# ---------------------------------------------------------------------------------
def _harmonic(k):
    return sum(1.0 / m for m in range(1, k + 1))


def two_over_x2_minus_k2(x):
    """2/x^2 - K2(x) for x > 0.

    x <= 2: series 1/2 + y * sum_k [ln(x/2) + gamma - (H_k + H_{k+2})/2] y^k/(k!(k+2)!),
    y = x^2/4 (A&S 9.6.11 with n = 2); x > 2: direct (no cancellation there).
    """
    x = float(x)
    if x > 2.0:
        return 2.0 / (x * x) - float(special.kv(2, x))
    y = 0.25 * x * x
    lx = math.log(0.5 * x) + EULER_GAMMA
    s = 0.0
    term = 1.0 / 2.0  # y^0/(0! 2!)
    k = 0
    while True:
        c = lx - 0.5 * (_harmonic(k) + _harmonic(k + 2))
        s += c * term
        k += 1
        term *= y / (k * (k + 2))
        if term < 1e-19 * max(1.0, abs(s)) and k > 3:
            break
    return 0.5 + y * s


def k0(x):
    """K0(x) for x > 0 (series A&S 9.6.13 for x <= 2, scipy otherwise)."""
    x = float(x)
    if x > 2.0:
        return float(special.k0(x))
    y = 0.25 * x * x
    i0 = 0.0
    tail = 0.0
    term = 1.0
    k = 0
    hk = 0.0
    while True:
        i0 += term
        tail += hk * term
        k += 1
        hk += 1.0 / k
        term *= y / (k * k)
        if term < 1e-19 and k > 3:
            break
    return -(math.log(0.5 * x) + EULER_GAMMA) * i0 + tail


def k2(x):
    x = float(x)
    return 2.0 / (x * x) - two_over_x2_minus_k2(x) if x <= 2.0 else float(special.kv(2, x))


def inv_x2_minus_w(x):
    """1/x^2 - (K0(x) + K2(x))/2 = (2/x^2 - K2)/2 - K0/2."""
    return 0.5 * two_over_x2_minus_k2(x) - 0.5 * k0(x)


def i0_minus_1(y):
    """I0(y) - 1 without cancellation for small y."""
    y = float(y)
    if y > 1.0:
        return float(special.i0(y)) - 1.0
    q = 0.25 * y * y
    s = 0.0
    term = q
    k = 1
    while term > 1e-20 * max(s, 1e-300):
        s += term
        k += 1
        term *= q / (k * k)
    return s


def i2(x):
    x = float(x)
    return float(special.iv(2, x))


# ---------------------------------------------------------------------------------
# radial integrals
# ---------------------------------------------------------------------------------
_QUAD = dict(epsabs=0.0, epsrel=2e-14, limit=500)


def _breaks_up(a, b, delta, alpha):
    """Break points for [a, b] (a >= 0): geometric away from 0 on the blob scale, no
    piece wider than 2/alpha (so exponential Bessel growth is resolved)."""
    pts = [a]
    x = a
    while x < b:
        w = max(x, 0.125 * delta)
        if alpha > 0:
            w = min(w, 2.0 / alpha)
        x = min(b, x + w)
        pts.append(x)
    return pts


def a1_integral(r, alpha, delta):
    """A1(r) = int_0^r (I0(alpha s) - 1) phi(s) s ds."""
    if r == 0.0:
        return 0.0
    f = lambda s: i0_minus_1(alpha * s) * float(blob(s, delta)) * s
    tot = 0.0
    pts = _breaks_up(0.0, r, delta, alpha)
    for lo, hi in zip(pts[:-1], pts[1:]):
        tot += integrate.quad(f, lo, hi, **_QUAD)[0]
    return tot


def c_integral(r, alpha, delta):
    """C(r) = int_r^inf K0(alpha s) phi(s) s ds (alpha > 0)."""
    f = lambda s: k0(alpha * s) * float(blob(s, delta)) * s
    s_end = min(1e6 * delta, r + 80.0 / alpha)
    tot = 0.0
    if r < 0.125 * delta:
        # K0 has a logarithmic branch point at s = 0: let quad's extrapolation handle it
        tot += integrate.quad(f, r, 0.125 * delta, **_QUAD)[0]
        start = 0.125 * delta
    else:
        start = r
    pts = _breaks_up(start, s_end, delta, alpha)
    for lo, hi in zip(pts[:-1], pts[1:]):
        tot += integrate.quad(f, lo, hi, **_QUAD)[0]
    return tot


# ---------------------------------------------------------------------------------
# kernel functions g1 = B'', g2 = (r B'' - B')/r^3
# ---------------------------------------------------------------------------------
def stokes_g(r, delta):
    """alpha = 0: the regularized Stokeslet with the same blob (Cortez 2001)."""
    r = np.asarray(r, dtype=np.float64)
    R = np.hypot(r, delta)
    g1 = (np.log(R + delta) - delta * (R + 2 * delta) / (R * (R + delta))) / (4 * np.pi)
    g2 = (R + 2 * delta) / (4 * np.pi * R * (R + delta) ** 2)
    return g1, g2


def singular_g(r, alpha):
    """delta -> 0 limit (singular Brinkmanlet): B0' = (a K1(a r) - 1/r)/(2 pi a^2),
    B0'' = (-a^2 K0 - a K1/r + 1/r^2)/(2 pi a^2)."""
    r = np.asarray(r, dtype=np.float64)
    x = alpha * r
    b1 = (alpha * special.k1(x) - 1.0 / r) / (2 * np.pi * alpha ** 2)
    b2 = (-alpha ** 2 * special.k0(x) - alpha * special.k1(x) / r + 1.0 / r ** 2) / (2 * np.pi * alpha ** 2)
    return b2, (r * b2 - b1) / r ** 3


def kernel_g(r, alpha, delta):
    """(g1, g2) at a single distance r >= 0, from the radial-integral definition."""
    r = float(r)
    if alpha == 0.0:
        g1, g2 = stokes_g(r, delta)
        return float(g1), float(g2)
    C = c_integral(r, alpha, delta)
    if r == 0.0:
        return -0.5 * C, (float(blob(0.0, delta)) - alpha * alpha * C) / 8.0
    x = alpha * r
    M = float(m0(r, delta))
    A = a1_integral(r, alpha, delta)
    w = 0.5 * (k0(x) + k2(x))
    g1 = inv_x2_minus_w(x) * M - w * A - 0.5 * (float(special.i0(x)) + i2(x)) * C
    g2 = (two_over_x2_minus_k2(x) * M - k2(x) * A - i2(x) * C) / (r * r)
    return g1, g2


def hankel_g(r, alpha, delta, kmax_over_delta=45.0):
    """Independent evaluation through the 2D Fourier transform (pins only).

    B^(k) = phi^(k)/(k^2 (k^2 + alpha^2)), phi^(k) = (1 + k d) e^{-k d}, so
    g1 = (1/2pi) int phi^ k/(k^2+a^2) (J1(kr)/(kr) - J0(kr)) dk,
    g2 = (1/(2 pi r^2)) int phi^ k/(k^2+a^2) J2(kr) dk.
    """
    phihat = lambda k: (1.0 + k * delta) * math.exp(-k * delta)
    kmax = kmax_over_delta / delta
    if r == 0.0:
        f1 = lambda k: phihat(k) * k / (k * k + alpha * alpha) * (-0.5)
        f2 = lambda k: phihat(k) * k / (k * k + alpha * alpha) * k * k / 8.0
        pts = sorted(set([0.0, 1.0 / delta, kmax] + ([alpha] if alpha > 0 else [])))
    else:
        def f1(k):
            z = k * r
            j = 0.5 - z * z / 16.0 if z < 1e-4 else special.j1(z) / z
            return phihat(k) * k / (k * k + alpha * alpha) * (j - special.j0(z))
        f2 = lambda k: phihat(k) * k / (k * k + alpha * alpha) * special.jv(2, k * r) / (r * r)
        step = math.pi / r
        n = int(kmax / step) + 1
        pts = sorted(set([0.0, kmax] + [min(kmax, i * step) for i in range(1, n + 1)] + ([alpha] if alpha > 0 else [])))
    g1 = g2 = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        if hi <= lo:
            continue
        g1 += integrate.quad(f1, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0]
        g2 += integrate.quad(f2, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0]
    return g1 / (2 * np.pi), g2 / (2 * np.pi)


def _node_values(r, alpha, delta):
    """(g1, g2) at ascending distances r > 0: A1 and C are accumulated from integrals
    between neighbouring points, then combined exactly as in :func:`kernel_g`."""
    if alpha == 0.0:
        return np.stack(stokes_g(r, delta), axis=1)
    fa = lambda s: i0_minus_1(alpha * s) * float(blob(s, delta)) * s
    fc = lambda s: k0(alpha * s) * float(blob(s, delta)) * s
    n = len(r)
    A = np.zeros(n)
    C = np.zeros(n)
    prev, acc = 0.0, 0.0
    for m in range(n):
        acc += integrate.quad(fa, prev, r[m], **_QUAD)[0]
        A[m] = acc
        prev = r[m]
    acc = c_integral(r[-1], alpha, delta)
    C[-1] = acc
    for m in range(n - 2, -1, -1):
        acc += integrate.quad(fc, r[m], r[m + 1], **_QUAD)[0]
        C[m] = acc
    out = np.zeros((n, 2))
    for m in range(n):
        x = alpha * r[m]
        M = float(m0(r[m], delta))
        w = 0.5 * (k0(x) + k2(x))
        out[m, 0] = inv_x2_minus_w(x) * M - w * A[m] - 0.5 * (float(special.i0(x)) + i2(x)) * C[m]
        out[m, 1] = (two_over_x2_minus_k2(x) * M - k2(x) * A[m] - i2(x) * C[m]) / (r[m] * r[m])
    return out


# ---------------------------------------------------------------------------------
# interpolation table over u = 1 + r^2/delta^2 (used by the oracle's time stepping)
# ---------------------------------------------------------------------------------
class KernelTable:
    """Piecewise Chebyshev interpolant of g1, g2 in u = 1 + r^2/delta^2.

    g1, g2 are even analytic functions of r whose only finite singularities in the
    complex r^2 plane are at r^2 = -delta^2, i.e. u = 0.  Octaves [2^e, 2^{e+1}) of u are
    cut into ``n_sub`` equal panels; each carries a degree-``deg`` Chebyshev series fitted
    at first-kind Chebyshev nodes from :func:`kernel_g`.  With n_sub = 4 the nearest
    singularity lies >= 9 half-widths from each panel centre, so degree 14 reaches
    rounding level.  Node values come from :func:`_node_values` (the integrals of
    :func:`kernel_g` accumulated between neighbouring nodes).  The pin test checks the
    table against pointwise evaluation.
    """

    def __init__(self, alpha, delta, r_max, n_sub=4, deg=14):
        self.alpha = float(alpha)
        self.delta = float(delta)
        u_max = 1.0 + (r_max / delta) ** 2
        self.n_oct = max(1, int(math.floor(math.log2(u_max))) + 1)
        self.n_sub = n_sub
        self.deg = deg
        npan = self.n_oct * n_sub
        self.coef = np.zeros((2, npan, deg + 1))
        t = np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))  # Chebyshev nodes
        # all nodes in ascending u; A1 and C accumulate integrals between neighbouring
        # nodes (the same integrals kernel_g evaluates from 0 / to infinity)
        us = []
        for e in range(self.n_oct):
            for j in range(n_sub):
                ua = 2.0 ** e * (1.0 + j / n_sub)
                ub = 2.0 ** e * (1.0 + (j + 1) / n_sub)
                us.append(np.sort(0.5 * (ua + ub) + 0.5 * (ub - ua) * t))
        u = np.concatenate(us)
        r = delta * np.sqrt(np.maximum(u - 1.0, 0.0))
        vals = _node_values(r, alpha, delta)
        for p in range(npan):
            vp = vals[p * (deg + 1):(p + 1) * (deg + 1)]
            tp = np.sort(t)
            for f in range(2):
                self.coef[f, p] = np.polynomial.chebyshev.chebfit(tp, vp[:, f], deg)

    def locate(self, u):
        u = np.asarray(u, dtype=np.float64)
        e = np.floor(np.log2(u)).astype(np.int64)
        e = np.clip(e, 0, self.n_oct - 1)
        base = 2.0 ** e
        j = np.clip(np.floor((u / base - 1.0) * self.n_sub).astype(np.int64), 0, self.n_sub - 1)
        ua = base * (1.0 + j / self.n_sub)
        w = base / self.n_sub
        t = 2.0 * (u - ua) / w - 1.0
        return e * self.n_sub + j, t

    def __call__(self, r):
        r = np.asarray(r, dtype=np.float64)
        u = 1.0 + (r / self.delta) ** 2
        p, t = self.locate(u)
        if np.any(u >= 2.0 ** self.n_oct):
            raise ValueError("distance beyond the table range")
        out = []
        for f in range(2):
            c = self.coef[f, p]  # (..., deg+1)
            # Clenshaw recurrence for sum_k c_k T_k(t)
            b1 = np.zeros_like(t)
            b2 = np.zeros_like(t)
            for k in range(self.deg, 0, -1):
                b1, b2 = 2.0 * t * b1 - b2 + c[..., k], b1
            out.append(t * b1 - b2 + c[..., 0])
        return out[0], out[1]
