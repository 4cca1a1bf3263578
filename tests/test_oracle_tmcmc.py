"""Pins of the oracle's TMCMC (Sec. 3.2, Algorithm 1) and of the surrogate MLP."""
import math

import numpy as np
import pytest

import synthetic
from oracle import mlp
from oracle import tmcmc as tm


def _toy(mean, sd):
    mean = np.asarray(mean)
    sd = np.asarray(sd)

    def loglik(th):
        th = np.atleast_2d(th)
        return -0.5 * np.sum(((th - mean) / sd) ** 2, axis=1)

    return loglik


def test_gaussian_toy_posterior():
    # uniform prior on a wide box x Gaussian likelihood -> posterior N(mean, sd^2) (closed form)
    mean = np.array([0.7, -1.2, 2.0])
    sd = np.array([0.3, 0.5, 0.2])
    lo, hi = np.full(3, -8.0), np.full(3, 8.0)
    B = 2048
    th0 = synthetic.prior_samples(11, lo, hi, B)
    theta, ll, log = tm.run(th0, _toy(mean, sd), lo, hi, 11,
                            randoms=lambda j: synthetic.stage_randoms(11, j, B, 3))
    assert log.q[-1] == 1.0
    assert len(log.q) > 3
    m = theta.mean(0)
    s = theta.std(0)
    # Monte-Carlo standard error of the mean over seeds is ~0.1 sd for B = 2048 (correlated
    # chains) and ~0.03 for the sd ratio: 3 standard errors each.  A wrong chain target
    # (f_j instead of f_{j+1}) widens the posterior by ~sqrt(q_{j+1}/q_j) and fails.
    assert np.all(np.abs(m - mean) < 0.3 * sd)
    assert np.all(np.abs(s / sd - 1) < 0.1)


def _box_gauss_log_evidence(mean, sd, lo, hi):
    # log of (1/V) * prod_i int_lo^hi exp(-((x - mean_i)/sd_i)^2 / 2) dx, exactly (erf)
    from scipy.special import erf

    mean, sd, lo, hi = (np.asarray(v, dtype=np.float64) for v in (mean, sd, lo, hi))
    one_d = sd * np.sqrt(np.pi / 2) * (erf((hi - mean) / (sd * np.sqrt(2))) - erf((lo - mean) / (sd * np.sqrt(2))))
    return float(np.sum(np.log(one_d)) - np.sum(np.log(hi - lo)))


def test_model_evidence_single_stage_is_the_prior_mean_of_the_likelihood():
    # a likelihood wide enough that q goes from 0 to 1 in one stage: log p(D|M) = log S_0, the
    # Monte-Carlo mean of the likelihood over prior draws (Sec. 3.2), against the exact integral
    mean = np.array([0.5, -1.0, 2.0])
    sd = np.array([6.0, 8.0, 10.0])
    lo, hi = np.full(3, -8.0), np.full(3, 8.0)
    B = 4096
    th0 = synthetic.prior_samples(3, lo, hi, B)
    _, _, log = tm.run(th0, _toy(mean, sd), lo, hi, 3, randoms=lambda j: synthetic.stage_randoms(3, j, B, 3))
    assert log.q == [1.0]
    exact = _box_gauss_log_evidence(mean, sd, lo, hi)
    ll = _toy(mean, sd)(th0)
    assert log.log_s[0] == pytest.approx(math.log(np.mean(np.exp(ll))), rel=1e-12)
    # Monte-Carlo error of the mean of B draws of a likelihood with COV < 1: below 1.6 %
    assert abs(log.log_s[0] - exact) < 0.03, (log.log_s[0], exact)


def test_model_evidence_of_the_gaussian_toy():
    # sum_j log S_j over a multi-stage run against the closed form.  Short Metropolis chains
    # leave each stage's samples slightly off f_j, so the estimate sits a little low (about
    # -0.3 in log here, a 25 % underestimate); a wrong weight or a dropped l_max term would be
    # off by orders of magnitude
    mean = np.array([0.7, -1.2, 2.0])
    sd = np.array([0.3, 0.5, 0.2])
    lo, hi = np.full(3, -8.0), np.full(3, 8.0)
    exact = _box_gauss_log_evidence(mean, sd, lo, hi)
    est = []
    for seed in range(30, 38):
        B = 2048
        th0 = synthetic.prior_samples(seed, lo, hi, B)
        _, _, log = tm.run(th0, _toy(mean, sd), lo, hi, seed, randoms=lambda j: synthetic.stage_randoms(seed, j, B, 3))
        assert len(log.q) > 2
        est.append(sum(log.log_s))
    assert abs(np.mean(est) - exact) < 0.6, (est, exact)


def test_delayed_acceptance_keeps_target():
    mean = np.array([0.3, 0.1])
    sd = np.array([0.2, 0.4])
    lo, hi = np.full(2, -5.0), np.full(2, 5.0)
    B = 2048
    exact = _toy(mean, sd)
    surrogate = _toy(mean + 0.05, sd * 1.2)  # deliberately biased screen
    th0 = synthetic.prior_samples(5, lo, hi, B)
    theta, _, log = tm.run(th0, exact, lo, hi, 5, surrogate_fn=surrogate,
                           randoms=lambda j: synthetic.stage_randoms(5, j, B, 2))
    assert np.all(np.abs(theta.mean(0) - mean) < 0.3 * sd)
    assert np.all(np.abs(theta.std(0) / sd - 1) < 0.12)


def test_q_solve_hits_cov_target():
    rng = np.random.default_rng(0)
    ll = rng.normal(-500, 40, size=1000)
    a = tm.analyze(rng.normal(size=(1000, 2)), ll, 0.0)
    assert 0 < a["q_next"] < 1
    assert abs(tm.cov_of_weights(ll, a["dq"]) - 1.0) < 1e-10
    # weights normalised, covariance symmetric positive definite
    assert abs(a["wbar"].sum() - 1) < 1e-14
    assert np.all(np.linalg.eigvalsh(a["sigma"]) > 0)


def test_q_reaches_one_when_weights_flat():
    ll = np.full(64, -3.0) + 1e-6 * np.arange(64)
    a = tm.analyze(np.zeros((64, 1)) + np.arange(64)[:, None], ll, 0.4)
    assert a["q_next"] == 1.0


def test_diverged_samples_have_zero_weight():
    ll = np.array([-1.0, -np.inf, -2.0, -np.inf])
    w, _ = tm._weights(ll, 0.5)
    assert w[1] == 0 and w[3] == 0 and w[0] == 1.0


def test_resample_against_brute_force():
    rng = np.random.default_rng(4)
    for B in (1, 3, 17, 64):
        w = rng.uniform(0, 1, B) ** 3
        w[rng.integers(0, B)] = 1.0
        if B > 2:
            w[0] = 0.0
        u = synthetic.uniforms(9, synthetic.RESAMPLE, B, B)
        idx = tm.resample(w, u)
        W = np.floor(w * 2.0 ** 40).astype(np.int64)
        tot = int(W.sum())
        for k in range(B):
            t = min(int(math.floor(u[k] * tot)), tot - 1)
            acc = 0
            for i in range(B):
                acc += int(W[i])
                if acc > t:
                    break
            assert idx[k] == i
        if B > 2:
            assert not np.any(idx == 0)  # zero weight never selected
        uniq, n_c, off = tm.chains(idx, B)
        assert n_c.sum() == B


def test_mlp_gradients_finite_difference():
    rng = np.random.default_rng(2)
    params = mlp.init_params(rng, (5, 7, 6, 4))
    x = rng.normal(size=(9, 5))
    t = rng.normal(size=(9, 4))
    grads = mlp.backward(params, x, t)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            Wp = [(a.copy(), c.copy()) for a, c in params]
            Wm = [(a.copy(), c.copy()) for a, c in params]
            Wp[li][0][i, j] += h
            Wm[li][0][i, j] -= h
            fd = (mlp.loss(Wp, x, t) - mlp.loss(Wm, x, t)) / (2 * h)
            assert abs(fd - grads[li][0][i, j]) < 1e-7 * max(1.0, abs(fd))
        Wp = [(a.copy(), c.copy()) for a, c in params]
        Wm = [(a.copy(), c.copy()) for a, c in params]
        Wp[li][1][0] += h
        Wm[li][1][0] -= h
        fd = (mlp.loss(Wp, x, t) - mlp.loss(Wm, x, t)) / (2 * h)
        assert abs(fd - grads[li][1][0]) < 1e-7 * max(1.0, abs(fd))


def test_gelu_derivative_and_values():
    x = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(x))) < 1e-8
    # GELU(x) = x Phi(x): Phi(1) = 0.8413447460685429
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15


def test_adam_step_textbook():
    p = [(np.array([[1.0]]), np.array([0.5]))]
    g = [(np.array([[0.2]]), np.array([-0.1]))]
    z = [(np.zeros((1, 1)), np.zeros(1))]
    p1, m1, v1 = mlp.adam_step(p, g, z, z, 1, lr=0.01)
    # first step: m_hat = g, v_hat = g^2 -> update = lr * g/(|g| + eps)
    assert abs(p1[0][0][0, 0] - (1.0 - 0.01 * 0.2 / (0.2 + 1e-8))) < 1e-15
    assert abs(p1[0][1][0] - (0.5 + 0.01 * 0.1 / (0.1 + 1e-8))) < 1e-15


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.0e-3, 65504.0])
    r = mlp.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0          # halfway, rounds to even
    assert r[2] == 1.0078125    # above halfway rounds up
    assert abs(r[3] / v[3] - 1) < 2 ** -8


def test_surrogate_loglik_reduces_to_the_gaussian_likelihood():
    """With all weights and biases zero the network outputs 0, so the surrogate predicts
    out_mean: its log-likelihood is then the Gaussian likelihood (Sec. 3.1) of that fixed
    trajectory.  With 80 observation rows and stride 2 the misfit over the 40 used rows is
    doubled, which is the full-record likelihood when both rows of each pair agree."""
    from oracle import mlp as om
    from oracle import swimmer as sw

    rng = np.random.default_rng(4)
    zero = [(np.zeros_like(W), np.zeros_like(b)) for W, b in om.init_params(rng)]
    lo, hi = [0.0, -1.0, 0.05, 3.0, 6.0], [10.0, 1.0, 0.2, 3.0, 6.0]
    theta = rng.uniform([0.0, -1.0, 0.05], [10.0, 1.0, 0.2], size=(5, 3))
    pred = rng.normal(size=80)
    D40 = pred.reshape(40, 2) + 0.01 * rng.normal(size=(40, 2))
    ll = om.surrogate_loglik(zero, theta, lo, hi, pred, np.ones(80), 1, 3.0, 6.0, D40, 0.02)
    ref = sw.log_likelihood(pred.reshape(40, 2), D40, 0.02)
    assert np.allclose(ll, ref, rtol=1e-13)
    D80 = np.repeat(D40, 2, axis=0)  # rows 1, 3, 5, ... are the ones used with stride 2
    ll2 = om.surrogate_loglik(zero, theta, lo, hi, pred, np.ones(80), 2, 3.0, 6.0, D80, 0.02)
    ref2 = sw.log_likelihood(np.repeat(pred.reshape(40, 2), 2, axis=0), D80, 0.02)
    assert np.allclose(ll2, ref2, rtol=1e-13)
    # a fourth unknown scales sigma per sample
    th4 = np.column_stack([theta, np.full(5, 0.5)])
    ll4 = om.surrogate_loglik(zero, th4, lo, hi, pred, np.ones(80), 1, 3.0, 6.0, D40, 0.04)
    assert np.allclose(ll4, ref, rtol=1e-13)
    # the inputs: box ends map to -1 and +1, an empty range to 0, rounded to FP32
    x = om.surrogate_inputs(np.array([[0.0, 1.0, 0.125]]), lo, hi, 3.0, 6.0)
    assert np.allclose(x, [[-1.0, 1.0, 0.0, 0.0, 0.0]], rtol=0, atol=1e-15)


def test_bf16_operand_mode_reduces_to_the_plain_network(monkeypatch):
    """The BF16-operand mode rounds the factors of the 256-wide layers' products and nothing
    else: with the rounding made the identity it is the plain FP64 network and gradient, and
    the first layer's inputs are never rounded."""
    from oracle import mlp as om

    rng = np.random.default_rng(8)
    P = [(W, rng.normal(0, 0.1, b.shape)) for W, b in om.init_params(rng)]
    x = rng.uniform(-1, 1, (6, 5))
    t = rng.normal(size=(6, 80))
    rounded_inputs = []
    real = om.bf16_round

    def spy(a):
        rounded_inputs.append(np.asarray(a).shape)
        return np.asarray(a, dtype=np.float64)

    monkeypatch.setattr(om, "bf16_round", spy)
    y1 = om.forward(P, x, bf16_operands=True)
    g1 = om.backward(P, x, t, bf16_operands=True)
    assert (6, 5) not in rounded_inputs  # the network inputs stay exact
    monkeypatch.setattr(om, "bf16_round", real)
    assert np.array_equal(y1, om.forward(P, x))
    for (a, b), (c, d) in zip(g1, om.backward(P, x, t)):
        assert np.array_equal(a, c) and np.array_equal(b, d)
    # with the real rounding the outputs move, by about the BF16 spacing
    y2 = om.forward(P, x, bf16_operands=True)
    assert 0 < np.max(np.abs(y2 - y1)) < 0.05 * np.max(np.abs(y1))


def test_plain_model_judges_the_surrogate():
    """The fallback rule of delayed acceptance: a surrogate that differs from the exact
    log-likelihood by a constant (the offset cancels in the screen's ratio) keeps screening at
    every stage; one whose error spreads over many nats is dropped as soon as a stage judges it
    above 1 nat at that stage's exponent, the stages after it run plain Metropolis, and the
    posterior is still the exact one (closed form)."""
    mean = np.array([0.3, 0.1])
    sd = np.array([0.2, 0.4])
    lo, hi = np.full(2, -5.0), np.full(2, 5.0)
    B = 2048
    exact = _toy(mean, sd)
    rnd = lambda j: synthetic.stage_randoms(6, j, B, 2)
    th0 = synthetic.prior_samples(6, lo, hi, B)
    _, _, good = tm.run(th0, exact, lo, hi, 6, surrogate_fn=lambda th: exact(th) - 3.0, randoms=rnd)
    assert all(good.surrogate_used) and max(good.surrogate_error) < 1e-9
    noisy = lambda th: exact(th) + 40.0 * np.sin(37.0 * np.atleast_2d(th)[:, 0])
    theta, _, bad = tm.run(th0, exact, lo, hi, 6, surrogate_fn=noisy, randoms=rnd)
    used, err = bad.surrogate_used, bad.surrogate_error
    assert used[0] and not all(used)
    assert all(used[j] == (err[j - 1] <= 1.0) for j in range(1, len(used)))
    assert np.all(np.abs(theta.mean(0) - mean) < 0.3 * sd)
    assert np.all(np.abs(theta.std(0) / sd - 1) < 0.12)
