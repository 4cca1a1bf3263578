"""The learned surrogate end to end on the GPU: trained by the library's own MLP kernels on
forward runs the forward kernel generates, then used as a delayed-acceptance screen inside
TMCMC.  Delayed acceptance keeps the exact target, so the posterior must agree with plain
TMCMC; the gain is the number of exact forward-model runs it saves."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1910_12007_gb300 as g  # noqa: E402
from paper_1910_12007_gb300 import surrogate as sg  # noqa: E402

DEV = torch.device("cuda:0")
LO = (0.0, -1.0, 0.05)
HI = (10.0, 1.0, 0.2)
TRUTH = (1.0, 0.0, 0.1)


def _cfg(b_max):
    return g.SwimmerConfig(n_max=12, b_max=b_max, length=1.0, dt=2e-4, steps=4000, obs_every=100,
                           precision=g.FP32C)


@pytest.fixture(scope="module")
def trained():
    h = g.swimmer_init(_cfg(1024))
    th_train = torch.tensor(synthetic.prior_samples(31, LO, HI, 6144), device=DEV)
    sur = sg.train(h, th_train, LO, HI, epochs=120, batch=512, lr=2e-3, seed=3)
    th_val = torch.tensor(synthetic.prior_samples(32, LO, HI, 512), device=DEV)
    traj, status = sg.generate_training_set(h, th_val)
    err = sg.validation_error(sur, traj, th_val, status)
    h.close()
    return sur, err


def test_surrogate_learns_the_forward_model(trained):
    sur, err = trained
    assert sur.losses[-1] < 0.05 * sur.losses[0]
    # relative to the spread of the head trajectories over the prior
    assert err < 0.08, err


def _run(sur, use_surrogate, B=512, seed=11):
    cfg = _cfg(B)
    h = g.swimmer_init(cfg)
    truth_traj, _, _ = g.forward_batch(h, torch.tensor([TRUTH], dtype=torch.float64, device=DEV))
    xi = truth_traj[0].cpu().numpy()
    sigma = 0.05 * float(np.mean(np.abs(xi)))
    D = xi + sigma * synthetic.normals(1234, synthetic.NOISE, 0, xi.size).reshape(xi.shape)
    obs = torch.tensor(D, device=DEV)
    if use_surrogate:
        sur.attach(h)
    th0 = torch.tensor(synthetic.prior_samples(seed, LO, HI, B), device=DEV)
    log = []
    st = g.tmcmc_run(h, th0, obs, sigma, LO, HI, lambda j: synthetic.stage_randoms(seed, j, B, 3),
                     use_surrogate=use_surrogate, log=log)
    torch.cuda.synchronize()
    out = st.theta.cpu().numpy(), log
    h.close()
    return out


def test_delayed_acceptance_matches_plain_and_saves_forward_runs(trained):
    sur, _ = trained
    th_plain, log_plain = _run(sur, False)
    th_da, log_da = _run(sur, True)
    assert log_plain[-1]["q"] == 1.0 and log_da[-1]["q"] == 1.0
    m_p, s_p = th_plain.mean(0), th_plain.std(0)
    m_d, s_d = th_da.mean(0), th_da.std(0)
    # same target: moments agree to Monte-Carlo accuracy of two correlated 512-sample runs
    assert np.all(np.abs(m_d - m_p) <= 0.02 * np.abs(m_p) + 0.5 * s_p), (m_d, m_p, s_p)
    assert np.all(np.abs(s_d - s_p) <= 0.5 * s_p), (s_d, s_p)
    # forward runs the chains needed (pre-fetched runs off the realized paths excluded)
    exact_plain = sum(s["n_exact_path"] for s in log_plain)
    exact_da = sum(s["n_exact_path"] for s in log_da)
    screened = sum(s["n_screened"] for s in log_da)
    acc_plain = sum(s["n_accept"] for s in log_plain) / exact_plain
    acc_da = sum(s["n_accept"] for s in log_da) / exact_da
    assert screened > 0
    # the gain: the screen removes proposals the exact model would reject, so fewer exact
    # forward runs are made and a larger share of them is accepted; the saving is about the
    # number of proposals plain TMCMC rejects at most (the two runs' chains differ, so allow
    # three standard deviations of that count)
    rejected_plain = exact_plain - sum(s["n_accept"] for s in log_plain)
    assert exact_da < exact_plain, (exact_da, exact_plain)
    assert exact_plain - exact_da <= rejected_plain + 3 * math.sqrt(rejected_plain)
    assert acc_da > acc_plain, (acc_da, acc_plain)


def test_a_run_from_the_prior_trusts_the_surrogate_anew(trained):
    """The plain model's judgement is state of the handle that carries over from stage to
    stage; a second run on the same handle starts from the prior and must not inherit the end
    of the first.  The trained surrogate's predictions are shifted by ten noise levels, which
    moves its log-likelihood by amounts that vary with theta by far more than 1 nat, so the
    first run ends with the surrogate distrusted."""
    import dataclasses

    sur, _ = trained
    B, seed = 256, 12
    h = g.swimmer_init(_cfg(B))
    truth_traj, _, _ = g.forward_batch(h, torch.tensor([TRUTH], dtype=torch.float64, device=DEV))
    xi = truth_traj[0].cpu().numpy()
    sigma = 0.01 * float(np.mean(np.abs(xi)))
    obs = torch.tensor(xi + sigma * synthetic.normals(1234, synthetic.NOISE, 0, xi.size).reshape(xi.shape),
                       device=DEV)
    dataclasses.replace(sur, out_mean=sur.out_mean + 10.0 * sigma).attach(h)
    th0 = torch.tensor(synthetic.prior_samples(seed, LO, HI, B), device=DEV)
    logs, thetas = [], []
    for _ in range(2):
        log = []
        st = g.tmcmc_run(h, th0, obs, sigma, LO, HI, lambda j: synthetic.stage_randoms(seed, j, B, 3),
                         use_surrogate=True, log=log)
        thetas.append(st.theta.cpu().numpy())
        logs.append(log)
    h.close()
    used = [s["surrogate_used"] for s in logs[0]]
    assert used[0] == 1 and not used[-1], used
    # the judged error sums over proposals in atomic order: equal to rounding
    err = [[s.pop("surrogate_error") for s in log] for log in logs]
    assert np.allclose(err[0], err[1], rtol=1e-9, equal_nan=True)
    assert logs[0] == logs[1]
    assert np.array_equal(thetas[0], thetas[1])


def test_delayed_acceptance_fp64_matches_oracle_sample_by_sample():
    """The two-stage Metropolis-Hastings chains of delayed acceptance (stage 1 on the
    surrogate, stage 2 on the exact model; Sec. 3.2, Algorithm 1 otherwise) on the FP64
    kernel against the oracle's, sample by sample, over a whole TMCMC run.  The network's
    weights are seeded inputs (not trained here), so both sides hold the same surrogate: a
    smooth function of theta that predicts the true trajectory plus a perturbation of half
    the noise level, whose log-likelihood varies by nats across the prior."""
    import multiprocessing as mp

    from oracle import mlp as om
    from oracle import swimmer as sw
    from oracle import tmcmc as tm

    base = sw.SwimmerParams(n=12, dt=2e-4, steps=5000, obs_every=125, alpha=1.0, amp=0.1)
    B, seed = 96, 44
    obs, _, _, st = sw.run_c_batch([base.with_theta(TRUTH)])
    xi = obs[0]
    sigma = sw.noise_sigma(xi, 0.05)
    D = xi + sigma * synthetic.normals(1234, synthetic.NOISE, 0, xi.size).reshape(xi.shape)
    # seeded network (BF16-rounded weights on both sides), output normalization around xi
    rng = np.random.default_rng(9)
    params = [(W, rng.normal(0, 0.1, size=b.shape)) for W, b in om.init_params(rng)]
    flat = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)
    rounded, o = [], 0
    for fi, fo in zip(om.LAYERS[:-1], om.LAYERS[1:]):
        W = flat[o:o + fo * fi].astype(np.float64).reshape(fo, fi)
        o += fo * fi
        rounded.append((om.bf16_round(W), flat[o:o + fo].astype(np.float64)))
        o += fo
    out_mean = xi.reshape(-1)
    out_std = np.full(80, 0.5 * sigma)
    log10_kt, omega = math.log10(base.k_t), base.omega
    in_lo = list(LO) + [log10_kt, omega]
    in_hi = list(HI) + [log10_kt, omega]
    # GPU: FP64 kernel, surrogate attached, delayed acceptance
    cfg = g.SwimmerConfig(n_max=base.n, b_max=B, length=base.length, dt=base.dt, steps=base.steps,
                          obs_every=base.obs_every, precision=g.FP64)
    h = g.swimmer_init(cfg)
    g.swimmer_surrogate_set(h, torch.tensor(flat, device=DEV), in_lo, in_hi, out_mean, out_std, 1, log10_kt, omega)
    th0 = synthetic.prior_samples(seed, LO, HI, B)
    log_g = []
    stg = g.tmcmc_run(h, torch.tensor(th0, device=DEV), torch.tensor(D, device=DEV), sigma, LO, HI,
                      lambda j: synthetic.stage_randoms(seed, j, B, 3), use_surrogate=True, log=log_g)
    torch.cuda.synchronize()
    th_g, ll_g = stg.theta.cpu().numpy(), stg.loglik.cpu().numpy()
    h.close()
    # oracle: the same chains with the oracle's surrogate and forward model
    surr_fn = lambda th: om.surrogate_loglik(rounded, th, in_lo, in_hi, out_mean, out_std, 1, log10_kt, omega, D,
                                             sigma)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count())) as pool:
        fn = lambda th: sw.batch_log_likelihood(base, th, D, sigma, pool=pool, chunk=4)
        th_o, ll_o, log_o = tm.run(th0, fn, LO, HI, seed, surrogate_fn=surr_fn,
                                   randoms=lambda j: synthetic.stage_randoms(seed, j, B, 3))
    assert len(log_g) == len(log_o.q) and len(log_g) >= 2
    assert [s["q"] for s in log_g] == pytest.approx(log_o.q, rel=1e-9)
    assert [s["unique"] for s in log_g] == log_o.unique
    # exact forward runs the one-step chains make, and accepted moves, stage by stage
    assert [s["n_exact_path"] for s in log_g] == log_o.n_exact
    # the plain model's judgement of the surrogate, and the screening it allows, stage by stage
    assert [bool(s["surrogate_used"]) for s in log_g] == log_o.surrogate_used
    err_g = np.array([s["surrogate_error"] for s in log_g])
    # the judged error is a standard deviation of l - l~ over the stage's proposals; the GPU's
    # l~ is FP32 MLP arithmetic on values of a few hundred nats (rounding near 1e-5 nats), and a
    # standard deviation moves by at most the largest change of its terms
    assert np.allclose(err_g, log_o.surrogate_error, rtol=0, atol=1e-4, equal_nan=True)
    assert [s["n_accept"] / B for s in log_g] == pytest.approx(log_o.accept, abs=0)
    assert np.allclose(th_g, th_o, rtol=1e-8, atol=1e-10)
    assert np.allclose(ll_g, ll_o, rtol=1e-8, atol=1e-8)
