"""Full sperm model (flagellum + circular head + neck), FP64 (oracle; test infrastructure only).

Model (Appendix; Table Tab:param)
---------------------------------
* Flagellum: the points X_0..X_{N_F-1} of ``oracle.swimmer`` (tension and bending energies
  Eqs. EFT, EFB with the same readings); X_{N_F-1} is the proximal end, joined to the head.
* Head: N_H (even) points on a circle of radius H_r, H_m = c + H_r (cos th_m, sin th_m),
  th_m = 2 pi m / N_H (counter-clockwise).  Initially the centre c sits on the line of the
  flagellum, H_r + dN to the right of its proximal point, so H_{N_H/2} (th = pi) faces the
  flagellum at distance dN.
* Head bending: E_HB = K_HC sum_m (kappa_m - 1/H_r)^2 ds_H, kappa_m the curvature of Eq.
  (curva) from periodic central differences, ds_H = 2 pi H_r / N_H (trapezoid rule on the
  closed curve).
* Head inextensibility: Hookean springs E = K_HT sum (l/l0 - 1)^2 l0 between membrane
  neighbours (m, m+1 mod N_H) and between points pi apart (m, m + N_H/2), rest lengths l0
  the initial lengths (the form of Eq. EFT, whose rest length is ds).
* Neck: five springs of the same form, stiffness K_NT, rest lengths the initial lengths:
  X_{N_F-1} to the head points at th = pi - dth, pi, pi + dth and X_{N_F-2} to th = pi +- dth.
* Neck angle: z1 = H(pi) - X_{N_F-1}, z2 = H(pi + dth) - H(pi - dth);
  E_NA = K_NA (z1 . z2)^2 (zero when the vectors are orthogonal, as initially).
* Forces F = -dE/dX (Eq. Fenergy), exact gradients; velocity Eq. (BrV) over all
  N_T = N_F + N_H points; forward Euler as in ``oracle.swimmer``.
* Observations (Sec. 4.1): head-centre velocity (x, y) estimated from the centre (mean of the
  head points) every ``obs_every`` steps: (c(t_o) - c(t_{o-1})) / (obs_every dt).

Readings where the paper is silent: H_r = N_H ds / (2 pi) (head points spaced like the
flagellum's), dN = ds, the unnormalised angle energy above, the circle counter-clockwise
from th = 0, delta = the Table's epsilon.  Pins (tests/test_oracle_sperm.py): forces against
central finite differences of the energy, zero net force and torque, springs and angle term at
rest initially, the flagellum-only model recovered when the head and neck are switched off,
first-order convergence in dt.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

from . import swimmer as sw


@dataclass(frozen=True)
class SpermParams:
    flag: sw.SwimmerParams          # flagellum, fluid and time stepping
    n_head: int = 24                # N_H (even)
    head_radius: float = 0.0        # H_r; 0 -> N_H ds / (2 pi)
    neck_gap: float = 0.0           # dN; 0 -> ds
    k_head_tens: float = 1e4        # K_{H,tens}
    k_head_c: float = 0.8           # K_{H,C}
    k_neck_tens: float = 500.0      # K_{N,tens}
    k_neck_ang: float = 1e4         # K_{N,ang}

    @property
    def nf(self):
        return self.flag.n

    @property
    def nt(self):
        return self.flag.n + self.n_head

    @property
    def hr(self):
        return self.head_radius if self.head_radius > 0 else self.n_head * self.flag.ds / (2 * math.pi)

    @property
    def gap(self):
        return self.neck_gap if self.neck_gap > 0 else self.flag.ds

    @property
    def ds_head(self):
        return 2 * math.pi * self.hr / self.n_head

    def with_theta(self, theta):
        return replace(self, flag=self.flag.with_theta(theta))


def initial_shape(p: SpermParams):
    Xf = sw.initial_shape(p.flag)
    end = Xf[-1]
    c = end + np.array([p.gap + p.hr, 0.0])
    th = 2 * math.pi * np.arange(p.n_head) / p.n_head
    H = c + p.hr * np.stack([np.cos(th), np.sin(th)], axis=1)
    return np.concatenate([Xf, H])


def head_index(p: SpermParams, m):
    return p.nf + (m % p.n_head)


def springs(p: SpermParams):
    """(i, j, stiffness) of every head, diametral and neck spring (rest length = initial)."""
    out = []
    nh, h2 = p.n_head, p.n_head // 2
    for m in range(nh):
        out.append((head_index(p, m), head_index(p, m + 1), p.k_head_tens))
    for m in range(h2):
        out.append((head_index(p, m), head_index(p, m + h2), p.k_head_tens))
    f1, f2 = p.nf - 1, p.nf - 2
    for dm in (-1, 0, 1):
        out.append((f1, head_index(p, h2 + dm), p.k_neck_tens))
    for dm in (-1, 1):
        out.append((f2, head_index(p, h2 + dm), p.k_neck_tens))
    X0 = initial_shape(p)
    return [(i, j, k, float(np.hypot(*(X0[j] - X0[i])))) for i, j, k in out]


def angle_points(p: SpermParams):
    """(flagellum end, H(pi), H(pi + dth), H(pi - dth)) point indices."""
    h2 = p.n_head // 2
    return p.nf - 1, head_index(p, h2), head_index(p, h2 + 1), head_index(p, h2 - 1)


def head_curvature(H, ds_h):
    """kappa_m from periodic central differences (Eq. curva on the closed head curve)."""
    xp, xm = np.roll(H, -1, axis=0), np.roll(H, 1, axis=0)
    a = (xp[:, 0] - xm[:, 0]) / (2 * ds_h)
    b = (xp[:, 1] - xm[:, 1]) / (2 * ds_h)
    c = (xp[:, 0] - 2 * H[:, 0] + xm[:, 0]) / ds_h ** 2
    d = (xp[:, 1] - 2 * H[:, 1] + xm[:, 1]) / ds_h ** 2
    return (a * d - b * c) / (a * a + b * b) ** 1.5


def energy(X, p: SpermParams, t):
    e = sw.energy(X[:p.nf], p.flag, t)
    for i, j, k, l0 in springs(p):
        ell = float(np.hypot(*(X[j] - X[i])))
        e += k * (ell / l0 - 1.0) ** 2 * l0
    kap = head_curvature(X[p.nf:], p.ds_head)
    e += p.k_head_c * float(np.sum((kap - 1.0 / p.hr) ** 2)) * p.ds_head
    f, hp, hplus, hminus = angle_points(p)
    z1, z2 = X[hp] - X[f], X[hplus] - X[hminus]
    e += p.k_neck_ang * float(z1 @ z2) ** 2
    return e


def forces(X, p: SpermParams, t):
    """F = -dE/dX, exact derivative of :func:`energy`."""
    F = np.zeros_like(X)
    F[:p.nf] = sw.forces(X[:p.nf], p.flag, t)
    for i, j, k, l0 in springs(p):
        d = X[j] - X[i]
        ell = float(np.hypot(*d))
        g = 2.0 * k * (ell / l0 - 1.0) * d / ell  # dE/dX_j
        F[j] -= g
        F[i] += g
    # head bending with periodic stencils (same chain rule as the flagellum's)
    H = X[p.nf:]
    h = p.ds_head
    xp, xm = np.roll(H, -1, axis=0), np.roll(H, 1, axis=0)
    a = (xp[:, 0] - xm[:, 0]) / (2 * h)
    b = (xp[:, 1] - xm[:, 1]) / (2 * h)
    cc = (xp[:, 0] - 2 * H[:, 0] + xm[:, 0]) / h ** 2
    dd = (xp[:, 1] - 2 * H[:, 1] + xm[:, 1]) / h ** 2
    S = a * a + b * b
    cross = a * dd - b * cc
    kap = cross * S ** -1.5
    ck = 2.0 * p.k_head_c * h * (kap - 1.0 / p.hr)
    z_a = dd * S ** -1.5 - 3.0 * a * cross * S ** -2.5
    z_b = -cc * S ** -1.5 - 3.0 * b * cross * S ** -2.5
    z_c = -b * S ** -1.5
    z_d = a * S ** -1.5
    G = np.zeros_like(H)
    # centre m depends on m-1 (via -a/2h, +c/h^2), m (-2c/h^2), m+1 (+a/2h, +c/h^2)
    gm = np.stack([-z_a / (2 * h) + z_c / h ** 2, -z_b / (2 * h) + z_d / h ** 2], axis=1)
    g0 = np.stack([-2.0 * z_c / h ** 2, -2.0 * z_d / h ** 2], axis=1)
    gp = np.stack([z_a / (2 * h) + z_c / h ** 2, z_b / (2 * h) + z_d / h ** 2], axis=1)
    G += np.roll(ck[:, None] * gm, -1, axis=0)  # centre m+1 acts on point m as its m-1 neighbour
    G += ck[:, None] * g0
    G += np.roll(ck[:, None] * gp, 1, axis=0)   # centre m-1 acts on point m as its m+1 neighbour
    F[p.nf:] -= G
    # neck angle: E = K (z1 . z2)^2
    f, hp, hplus, hminus = angle_points(p)
    z1, z2 = X[hp] - X[f], X[hplus] - X[hminus]
    w = 2.0 * p.k_neck_ang * float(z1 @ z2)
    F[hp] -= w * z2
    F[f] += w * z2
    F[hplus] -= w * z1
    F[hminus] += w * z1
    return F


def head_centre(X, p: SpermParams):
    return X[p.nf:].mean(axis=0)


def kernel_table(p: SpermParams):
    from .brinkmanlet import KernelTable

    return KernelTable(p.flag.alpha, p.flag.delta, 1.25 * (p.flag.length + p.gap + 2 * p.hr))


def run_numpy(p: SpermParams, table=None, steps=None, observe="velocity"):
    """Forward Euler time loop.  Returns (obs[n_obs, 2], X_final, status) with status 0 = ok,
    1 = diverged (non-finite, or a point moving more than ds).  ``observe``: "velocity" for
    head-centre velocities, "point" for the proximal flagellum point X_{N_F-1}."""
    fp = p.flag
    table = table or kernel_table(p)
    steps = fp.steps if steps is None else steps
    X = initial_shape(p)
    c_prev = head_centre(X, p)
    obs = []
    for n in range(steps):
        F = forces(X, p, n * fp.dt)
        v = sw.velocity(X, F, table, fp.mu)
        if not np.all(np.isfinite(v)) or np.max(np.abs(v)) * fp.dt > fp.ds:
            return np.array(obs).reshape(-1, 2), X, 1
        X = X + fp.dt * v
        if (n + 1) % fp.obs_every == 0:
            if observe == "velocity":
                c = head_centre(X, p)
                obs.append((c - c_prev) / (fp.obs_every * fp.dt))
                c_prev = c
            else:
                obs.append(X[p.nf - 1].copy())
    return np.array(obs).reshape(-1, 2), X, 0


def mean_speed(X0, X1, p: SpermParams, T):
    """Head-centre x-displacement over the run divided by its duration."""
    return float(head_centre(X1, p)[0] - head_centre(X0, p)[0]) / T


# ---------------------------------------------------------------------------------------
# Two swimmers (Sec. 4.2): the same swimmer twice, the second displaced by d along y; each
# has its own elastic energy, the fluid couples them through the pair sum over all points.
# Observations: the distance between the last points of the tails (flagellum point 0) and
# between the head centres, every obs_every steps.
# ---------------------------------------------------------------------------------------
@dataclass(frozen=True)
class PairParams:
    one: SpermParams
    d: float = 2.0  # initial vertical separation of the two swimmers

    @property
    def nt(self):
        return 2 * self.one.nt


def pair_initial_shape(q: PairParams):
    X = initial_shape(q.one)
    return np.concatenate([X, X + np.array([0.0, q.d])])


def pair_forces(X, q: PairParams, t):
    n = q.one.nt
    return np.concatenate([forces(X[:n], q.one, t), forces(X[n:], q.one, t)])


def pair_energy(X, q: PairParams, t):
    n = q.one.nt
    return energy(X[:n], q.one, t) + energy(X[n:], q.one, t)


def pair_distances(X, q: PairParams):
    """(tail-tip distance, head-centre distance)."""
    n = q.one.nt
    tail = float(np.hypot(*(X[n] - X[0])))
    head = float(np.hypot(*(head_centre(X[n:], q.one) - head_centre(X[:n], q.one))))
    return np.array([tail, head])


def pair_kernel_table(q: PairParams):
    from .brinkmanlet import KernelTable

    p = q.one
    return KernelTable(p.flag.alpha, p.flag.delta, 1.25 * (p.flag.length + p.gap + 2 * p.hr + q.d))


def pair_run_numpy(q: PairParams, table=None, steps=None):
    """Forward Euler for both swimmers.  Returns (obs[n_obs, 2] = (tail, head) distances,
    X_final, status)."""
    fp = q.one.flag
    table = table or pair_kernel_table(q)
    steps = fp.steps if steps is None else steps
    X = pair_initial_shape(q)
    obs = []
    for n in range(steps):
        F = pair_forces(X, q, n * fp.dt)
        v = sw.velocity(X, F, table, fp.mu)
        if not np.all(np.isfinite(v)) or np.max(np.abs(v)) * fp.dt > fp.ds:
            return np.array(obs).reshape(-1, 2), X, 1
        X = X + fp.dt * v
        if (n + 1) % fp.obs_every == 0:
            obs.append(pair_distances(X, q))
    return np.array(obs).reshape(-1, 2), X, 0


def log_likelihood_two_sigma(obs_model, data, sigma_t, sigma_h):
    """Sec. 4.2, two noise levels: Sigma diagonal with sigma_t^2 on the tail distances (odd
    positions, 1-based) and sigma_h^2 on the head distances (even positions)."""
    r = np.asarray(data, dtype=np.float64).reshape(-1, 2) - np.asarray(obs_model, dtype=np.float64).reshape(-1, 2)
    m = r.shape[0]
    return (-0.5 * m * (math.log(2 * math.pi * sigma_t ** 2) + math.log(2 * math.pi * sigma_h ** 2))
            - 0.5 * float(np.sum(r[:, 0] ** 2)) / sigma_t ** 2 - 0.5 * float(np.sum(r[:, 1] ** 2)) / sigma_h ** 2)
