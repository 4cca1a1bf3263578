"""Elastic 2D flagellum forward model, FP64 (oracle; test infrastructure only).

Model (Appendix; Sec. 2.1; Sec. 3.1)
------------------------------------
* Points X_k, k = 0..N-1, spacing ds = L/(N-1), arclength s_k = k ds; k = 0 is the free
  distal end, k = N-1 the proximal ("head") end.  Initially straight: X_k = (s_k, 0).
* Preferred shape (Appendix): y^(s,t) = a (1 - s/L) sin(eta s - omega t); preferred
  curvature zeta^ = d^2 y^/ds^2 (Eq. curva, left)
      = -a [ (2 eta/L) cos(eta s - omega t) + (1 - s/L) eta^2 sin(eta s - omega t) ].
* Bending energy, Eq. (EFB): E_B = K_C sum_{k=1}^{N-2} (zeta_k - zeta^_k)^2 ds with the
  full nonlinear signed curvature of Eq. (curva, right) from central differences
  x' = (x_{k+1} - x_{k-1})/(2 ds), x'' = (x_{k+1} - 2 x_k + x_{k-1})/ds^2 (the paper's
  "second order finite differences", trapezoid weights 1 on interior points).
* Tension energy, Eq. (EFT) read as Hookean springs of rest length ds (the text after
  it): E_T = K_T sum_{k=0}^{N-2} (|X_{k+1} - X_k|/ds - 1)^2 ds.
* Forces, Eq. (Fenergy): F = -dE/dX, the exact gradient of the discrete energy.
* Velocity, Eq. (BrV): v_i = (1/mu) sum_j [ -F_j g1(r_ij) + (F_j . d_ij) d_ij g2(r_ij) ],
  d_ij = X_i - X_j, self term included (g1(0), d = 0).
* Time stepping (Appendix, last paragraph): forward Euler X^{n+1} = X^n + dt v(X^n, t_n).
* Observations: head point X_{N-1} after every ``obs_every`` steps.
* Likelihood, Eqs. (likelihood, fitness) with Sigma = sigma^2 I:
  log p = -(m/2) ln(2 pi sigma^2) - J/2, J = |D - g|^2/sigma^2.

Parity pins (tests/test_oracle_swimmer.py): forces against central finite differences
of the energy, zero net force and torque, the straight filament at a = 0 staying exactly
at rest, mirror symmetry, first-order convergence in dt, the C time loop against the
numpy time loop, the likelihood against a hand computation.  The end-to-end swimming
trajectory itself is "parity unpinned": the paper prints no trajectory for these settings.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, replace

import numpy as np

from .brinkmanlet import KernelTable


@dataclass(frozen=True)
class SwimmerParams:
    """Physical and numerical parameters of one forward run (Table Tab:param fields)."""

    n: int = 64                 # points on the flagellum
    length: float = 1.0         # flagellum length L (nondimensional)
    mu: float = 1.0             # viscosity
    delta_over_ds: float = 1.5  # blob width in units of ds
    dt: float = 1.25e-5         # forward Euler step
    k_t: float = 1e3            # tension stiffness K_T
    k_c: float = 1.0            # curvature stiffness K_C
    eta: float = 2 * math.pi    # wavenumber
    omega: float = 2 * math.pi  # angular frequency
    amp: float = 0.1            # amplitude a
    alpha: float = 1.0          # Brinkman resistance
    steps: int = 80000
    obs_every: int = 800

    @property
    def ds(self):
        return self.length / (self.n - 1)

    @property
    def delta(self):
        return self.delta_over_ds * self.ds

    @property
    def n_obs(self):
        return self.steps // self.obs_every

    def with_theta(self, theta):
        """theta = (alpha, log10 K_C, amplitude), the unknowns of the TMCMC problem."""
        return replace(self, alpha=float(theta[0]), k_c=10.0 ** float(theta[1]), amp=float(theta[2]))


def initial_shape(p: SwimmerParams):
    x = np.arange(p.n, dtype=np.float64) * p.ds
    return np.stack([x, np.zeros(p.n)], axis=1)


def preferred_curvature(p: SwimmerParams, t):
    """zeta^_k(t) at interior points k = 1..N-2 (second s-derivative of y^)."""
    s = np.arange(1, p.n - 1, dtype=np.float64) * p.ds
    ph = p.eta * s - p.omega * t
    return -p.amp * (2.0 * p.eta / p.length * np.cos(ph) + (1.0 - s / p.length) * p.eta ** 2 * np.sin(ph))


def curvature(X, ds):
    """Signed curvature zeta_k at interior points from central differences (Eq. curva)."""
    x, y = X[:, 0], X[:, 1]
    a = (x[2:] - x[:-2]) / (2 * ds)
    b = (y[2:] - y[:-2]) / (2 * ds)
    c = (x[2:] - 2 * x[1:-1] + x[:-2]) / ds ** 2
    d = (y[2:] - 2 * y[1:-1] + y[:-2]) / ds ** 2
    return (a * d - b * c) / (a * a + b * b) ** 1.5


def energy(X, p: SwimmerParams, t):
    """E = E_tension + E_bend (Eqs. EFT, EFB), discrete sums as in the module docstring."""
    ds = p.ds
    seg = np.diff(X, axis=0)
    ell = np.hypot(seg[:, 0], seg[:, 1])
    e_t = p.k_t * np.sum((ell / ds - 1.0) ** 2) * ds
    e_b = p.k_c * np.sum((curvature(X, ds) - preferred_curvature(p, t)) ** 2) * ds
    return e_t + e_b


def forces(X, p: SwimmerParams, t):
    """F = -dE/dX (Eq. Fenergy), exact derivative of :func:`energy`."""
    ds = p.ds
    n = p.n
    F = np.zeros_like(X)
    # tension: d/dX_{k+1} K_T ds (l/ds - 1)^2 = 2 K_T (l/ds - 1) t_hat
    seg = np.diff(X, axis=0)
    ell = np.hypot(seg[:, 0], seg[:, 1])
    tens = 2.0 * p.k_t * (ell / ds - 1.0)
    g = (tens / ell)[:, None] * seg
    F[1:] -= g
    F[:-1] += g
    # bending: c_k = 2 K_C ds (zeta_k - zeta^_k); zeta = (a d - b c) S^{-3/2}, S = a^2+b^2
    x, y = X[:, 0], X[:, 1]
    a = (x[2:] - x[:-2]) / (2 * ds)
    b = (y[2:] - y[:-2]) / (2 * ds)
    cc = (x[2:] - 2 * x[1:-1] + x[:-2]) / ds ** 2
    dd = (y[2:] - 2 * y[1:-1] + y[:-2]) / ds ** 2
    S = a * a + b * b
    cross = a * dd - b * cc
    zeta = cross * S ** -1.5
    ck = 2.0 * p.k_c * ds * (zeta - preferred_curvature(p, t))
    z_a = dd * S ** -1.5 - 3.0 * a * cross * S ** -2.5
    z_b = -cc * S ** -1.5 - 3.0 * b * cross * S ** -2.5
    z_c = -b * S ** -1.5
    z_d = a * S ** -1.5
    # chain rule through the stencils (k-1, k, k+1) -> array offsets (0, 1, 2)
    gx_m = -z_a / (2 * ds) + z_c / ds ** 2
    gx_0 = -2.0 * z_c / ds ** 2
    gx_p = z_a / (2 * ds) + z_c / ds ** 2
    gy_m = -z_b / (2 * ds) + z_d / ds ** 2
    gy_0 = -2.0 * z_d / ds ** 2
    gy_p = z_b / (2 * ds) + z_d / ds ** 2
    F[:-2, 0] -= ck * gx_m
    F[1:-1, 0] -= ck * gx_0
    F[2:, 0] -= ck * gx_p
    F[:-2, 1] -= ck * gy_m
    F[1:-1, 1] -= ck * gy_0
    F[2:, 1] -= ck * gy_p
    return F


def velocity(X, F, table, mu=1.0):
    """v_i = (1/mu) sum_j [-F_j g1(r_ij) + (F_j . d_ij) d_ij g2(r_ij)]  (Eq. BrV)."""
    d = X[:, None, :] - X[None, :, :]
    r = np.hypot(d[..., 0], d[..., 1])
    g1, g2 = table(r)
    fd = np.einsum("jc,ijc->ij", F, d)
    v = -np.einsum("ij,jc->ic", g1, F) + np.einsum("ij,ij,ijc->ic", fd, g2, d)
    return v / mu


def kernel_table(p: SwimmerParams, margin=1.25):
    """The oracle's interpolation table of g1, g2 for this run's (alpha, delta)."""
    return KernelTable(p.alpha, p.delta, margin * p.length)


def run_numpy(p: SwimmerParams, table=None, steps=None):
    """Forward Euler time loop in plain numpy (slow; small cases and cross-checks).

    Returns (obs[n_obs, 2], X_final[N, 2], status) with status 0 = ok, 1 = diverged
    (non-finite, or a point moving more than ds in one step)."""
    table = table or kernel_table(p)
    steps = p.steps if steps is None else steps
    X = initial_shape(p)
    obs = []
    for n in range(steps):
        F = forces(X, p, n * p.dt)
        v = velocity(X, F, table, p.mu)
        if not np.all(np.isfinite(v)) or np.max(np.abs(v)) * p.dt > p.ds:
            return np.array(obs).reshape(-1, 2), X, 1
        X = X + p.dt * v
        if (n + 1) % p.obs_every == 0:
            obs.append(X[-1].copy())
    return np.array(obs).reshape(-1, 2), X, 0


def log_likelihood(obs_model, data, sigma):
    """log p(D|theta) = -(m/2) ln(2 pi sigma^2) - J/2, J = sum (D - g)^2 / sigma^2."""
    r = np.asarray(data, dtype=np.float64).ravel() - np.asarray(obs_model, dtype=np.float64).ravel()
    m = r.size
    return -0.5 * m * math.log(2 * math.pi * sigma * sigma) - 0.5 * float(np.sum(r * r)) / (sigma * sigma)


def noise_sigma(truth_obs, gamma):
    """sigma = gamma * beta with beta the mean magnitude of the model outputs (Sec. 4)."""
    return gamma * float(np.mean(np.abs(truth_obs)))


def mean_speed(X0, X1, T):
    """Signed x-displacement of the centroid over the run divided by its duration."""
    return (float(np.mean(X1[:, 0])) - float(np.mean(X0[:, 0]))) / T


# ---------------------------------------------------------------------------------
# linear stability of forward Euler about the straight filament
# ---------------------------------------------------------------------------------
def euler_lambda_max(p: SwimmerParams, table=None, h=1e-6):
    """Largest real part of the eigenvalues of M H at the straight filament, where M is
    the Brinkmanlet mobility matrix and H the Hessian of the elastic energy (a = 0).
    Forward Euler is stable for dt * lambda_max < 2."""
    q = replace(p, amp=0.0)
    table = table or kernel_table(q)
    X = initial_shape(q)
    n = 2 * q.n
    H = np.zeros((n, n))
    for c in range(n):
        Xp = X.copy().ravel()
        Xm = X.copy().ravel()
        Xp[c] += h
        Xm[c] -= h
        H[:, c] = -(forces(Xp.reshape(-1, 2), q, 0.0) - forces(Xm.reshape(-1, 2), q, 0.0)).ravel() / (2 * h)
    H = 0.5 * (H + H.T)
    d = X[:, None, :] - X[None, :, :]
    r = np.hypot(d[..., 0], d[..., 1])
    g1, g2 = table(r)
    M = np.zeros((q.n, 2, q.n, 2))
    for a in range(2):
        for b in range(2):
            M[:, a, :, b] = (-g1 * (a == b) + g2 * d[..., a] * d[..., b]) / q.mu
    ev = np.linalg.eigvals(M.reshape(n, n) @ H)
    return float(np.max(ev.real))


# ---------------------------------------------------------------------------------
# the C time loop (same arithmetic, plain loops; built by oracle/build.py)
# ---------------------------------------------------------------------------------
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(os.path.dirname(__file__), "_oracle_forward.so")
        if not os.path.exists(path):
            from .build import build
            build()
        lib = ctypes.CDLL(path)
        d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
        P = ctypes.POINTER
        lib.oracle_forward_batch.argtypes = [
            i, P(i), P(d), d, d, d, d, d, d, l, l,          # B, n[], L[], mu, delta/ds, dt, K_T, eta, omega, steps, obs_every
            P(d), P(d), P(d),                              # alpha[], K_C[], amp[]
            i, i, P(i), P(d),                              # n_sub, deg, n_oct[], coef (concatenated)
            P(l), P(d), P(d), P(d), P(i),                  # coef offsets, obs[B, n_obs, 2], X_final[B, n_max, 2], xc[B, 2], status[B]
            i]                                             # threads
        lib.oracle_forward_batch.restype = i
        _LIB = lib
    return _LIB


def run_c_batch(params_list, tables=None, threads=0, steps=None):
    """Run several forward models through the C loop (OpenMP over samples).

    All runs share mu, delta/ds, dt, K_T, eta, omega, steps and obs_every; they may
    differ in n, L, alpha, K_C and amp.  Returns (obs[B, n_obs, 2], X_final list, xc[B, 2]
    = centroid x at start and end, status[B])."""
    lib = _lib()
    p0 = params_list[0]
    steps = p0.steps if steps is None else steps
    B = len(params_list)
    tables = tables or [kernel_table(p) for p in params_list]
    n_arr = np.array([p.n for p in params_list], dtype=np.int32)
    n_max = int(n_arr.max())
    coefs = [np.ascontiguousarray(t.coef) for t in tables]
    offs = np.cumsum([0] + [c.size for c in coefs[:-1]]).astype(np.int64)
    coef = np.ascontiguousarray(np.concatenate([c.ravel() for c in coefs]))
    n_oct = np.array([t.n_oct for t in tables], dtype=np.int32)
    n_obs = steps // p0.obs_every
    obs = np.zeros((B, max(n_obs, 1), 2))
    Xf = np.zeros((B, n_max, 2))
    xc = np.zeros((B, 2))
    status = np.zeros(B, dtype=np.int32)
    alpha = np.array([p.alpha for p in params_list])
    kc = np.array([p.k_c for p in params_list])
    amp = np.array([p.amp for p in params_list])
    lens = np.array([p.length for p in params_list])
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
    rc = lib.oracle_forward_batch(
        B, P(n_arr, i), P(lens, d), p0.mu, p0.delta_over_ds, p0.dt, p0.k_t, p0.eta, p0.omega,
        steps, p0.obs_every, P(alpha, d), P(kc, d), P(amp, d),
        tables[0].n_sub, tables[0].deg, P(n_oct, i), P(coef, d), P(offs, l),
        P(obs, d), P(Xf, d), P(xc, d), P(status, i), threads)
    if rc != 0:
        raise RuntimeError(f"oracle_forward_batch failed: {rc}")
    return obs[:, :n_obs], [Xf[b, : n_arr[b]] for b in range(B)], xc, status


# ---------------------------------------------------------------------------------
# many samples at once: tables + C loop in a spawn-started process pool
# ---------------------------------------------------------------------------------
def _loglik_chunk(args):
    base, thetas, D, sigma = args
    ps = [base.with_theta(t) for t in thetas]
    obs, _, _, st = run_c_batch(ps, threads=1)
    out = np.full(len(ps), -np.inf)
    for b in range(len(ps)):
        # a fourth column is the sample's noise level in units of sigma (sigma/beta inferred)
        sg = sigma * thetas[b][3] if len(thetas[b]) > 3 else sigma
        if st[b] == 0 and sg > 0:
            out[b] = log_likelihood(obs[b], D, sg)
    return out


def batch_log_likelihood(base: SwimmerParams, thetas, D, sigma, pool=None, chunk=8):
    """log p(D|theta) for every row of thetas (diverged runs give -inf).  ``pool`` is a
    multiprocessing pool created with the 'spawn' start method (or None: serial)."""
    thetas = np.asarray(thetas, dtype=np.float64)
    parts = [(base, thetas[i:i + chunk], D, sigma) for i in range(0, len(thetas), chunk)]
    res = pool.map(_loglik_chunk, parts) if pool is not None else [_loglik_chunk(a) for a in parts]
    return np.concatenate(res) if res else np.zeros(0)


# ---------------------------------------------------------------------------------------
# flow and pressure at target points (Eqs. BrP, BrV with targets x other than the swimmer)
# ---------------------------------------------------------------------------------------
def pressure_kernel(r, delta):
    """G_delta'(r)/r = M0(r)/r^2 (text after Eq. BrV), finite at r = 0: with R = sqrt(r^2 +
    delta^2), M0/r^2 = (R^2 + R delta + delta^2) / (2 pi R^3 (R + delta))."""
    r = np.asarray(r, dtype=np.float64)
    R = np.hypot(r, delta)
    return (R * R + R * delta + delta * delta) / (2.0 * np.pi * R ** 3 * (R + delta))


def flow_field(X, F, grid, table, delta, mu=1.0):
    """Velocity v(x) (Eq. BrV) and pressure p(x) = sum_j F_j . grad G_delta(|x - X_j|)
    (Eq. BrP) at the target points grid [G, 2], from point forces F [N, 2] at X [N, 2]."""
    grid = np.asarray(grid, dtype=np.float64)
    d = grid[:, None, :] - X[None, :, :]
    r = np.hypot(d[..., 0], d[..., 1])
    g1, g2 = table(r)
    fd = np.einsum("jc,gjc->gj", F, d)
    v = (-np.einsum("gj,jc->gc", g1, F) + np.einsum("gj,gj,gjc->gc", fd, g2, d)) / mu
    p = np.sum(fd * pressure_kernel(r, delta), axis=1)
    return v, p
