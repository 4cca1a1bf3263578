"""The oracle against constants the paper prints (tests/golden/paper_constants.txt, each
line with its citation).  The paper prints no worked-example output of the flagellum model
alone (its result tables are for the full sperm model with head and neck), so these pins are
the printed constants; the remaining pins are closed forms and invariants (the other oracle
test files)."""
import math
import os

import numpy as np
from scipy import integrate

from oracle import brinkmanlet as bk
from oracle import swimmer as sw
from oracle import tmcmc as tm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def _load():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, value, cite = line.split(None, 2)
        assert cite  # every value carries its citation
        vals[name] = float(value)
    return vals


P = _load()


def test_blob_moment_matches_the_printed_normalisation():
    for delta in (0.045, 0.0118, 0.3):
        val, err = integrate.quad(lambda r: r * bk.blob(r, delta), 0.0, np.inf, epsabs=0, epsrel=2e-14,
                                  limit=200)
        assert abs(val - P["blob_moment"]) <= 1e-12


def test_tmcmc_constants_are_the_printed_ones():
    assert tm.COV_TARGET == P["tmcmc_cov_target"]
    assert tm.B_SCALE == P["tmcmc_b"]
    # q starts at 0 and the last stage is run at q = 1 (Gaussian-toy run, small B)
    mean, sd = np.array([0.2, -0.4]), np.array([0.3, 0.2])

    def ll(th):
        th = np.atleast_2d(th)
        return -0.5 * np.sum(((th - mean) / sd) ** 2, axis=1)

    lo, hi = np.full(2, -5.0), np.full(2, 5.0)
    rng = np.random.default_rng(3)
    B = 256
    th0 = rng.uniform(lo, hi, size=(B, 2))

    def randoms(j):
        r = np.random.default_rng(100 + j)
        return r.uniform(size=B), r.uniform(size=(2, B)), r.standard_normal((B, 2))

    a0 = tm.analyze(th0, ll(th0), P["tmcmc_q0"])
    assert 0.0 < a0["q_next"] <= 1.0
    _, _, log = tm.run(th0, ll, lo, hi, 3, randoms=randoms)
    assert log.q[-1] == P["tmcmc_q_final"]
    assert all(b > a for a, b in zip(log.q, log.q[1:]))


def test_printed_time_step_exceeds_the_euler_bound_of_the_printed_flagellum():
    # reading of the forward-Euler stability: with the printed flagellum parameters the
    # printed time step is beyond dt * lambda_max < 2, so the configurations use smaller steps
    n = int(P["param_n_flagellum"])
    p = sw.SwimmerParams(n=n, length=1.0, delta_over_ds=P["param_epsilon"] * (n - 1), k_t=P["param_k_tens"],
                         k_c=P["param_k_c"], eta=P["param_eta"], omega=P["param_omega"], amp=P["param_amp"],
                         alpha=1.0, dt=P["param_dt"], steps=1, obs_every=1)
    assert math.isclose(p.delta, P["param_epsilon"], rel_tol=1e-12)
    lam = sw.euler_lambda_max(p)
    assert P["param_dt"] * lam > 2.0
    assert 1e-4 / 8 * lam < 2.0  # three halvings restore stability
