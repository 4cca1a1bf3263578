"""GPU parity of the TMCMC stage kernels (Sec. 3.2, Algorithm 1) against the oracle,
through the C ABI.  Resample indices are compared bit for bit; the annealing solve and
statistics to FP64 rounding; a whole TMCMC run on a small swimmer problem sample by
sample (FP64 path) and by posterior moments (FP32-compensated path)."""
import math
import multiprocessing as mp
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic
from oracle import swimmer as sw
from oracle import tmcmc as tm

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1910_12007_gb300 as g  # noqa: E402

DEV = torch.device("cuda:0")


def _h(b_max, **kw):
    cfg = g.SwimmerConfig(n_max=12, b_max=b_max, steps=10, obs_every=1)
    for k, v in kw.items():
        setattr(cfg, k, v)
    return g.swimmer_init(cfg)


@pytest.mark.parametrize("B,q", [(1000, 0.0), (777, 0.3), (64, 0.9), (4096, 0.05)])
def test_analyze_matches_oracle(B, q):
    rng = np.random.default_rng(B)
    ll = rng.normal(-300, 30, size=B)
    ll[rng.integers(0, B, size=B // 50)] = -np.inf
    th = rng.normal(size=(B, 3)) * [0.5, 0.3, 0.05] + [1.0, 0.0, 0.1]
    a = tm.analyze(th, ll, q)
    h = _h(B)
    w, st = g.tmcmc_analyze(h, torch.tensor(th, device=DEV), torch.tensor(ll, device=DEV), q)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    # layout: dq, q_next, log S, l_max, mu[4], Sigma[4][4], L[4][4], status (3 unknowns used)
    assert st[40] == 0.0
    assert abs(st[0] - a["dq"]) <= 1e-12 * max(a["dq"], 1e-300)
    assert st[1] == pytest.approx(a["q_next"], rel=1e-12)
    assert st[2] == pytest.approx(a["log_s"], rel=1e-12)
    assert np.allclose(st[4:7], a["mu"], rtol=1e-11, atol=1e-14)
    assert np.allclose(st[8:24].reshape(4, 4)[:3, :3], a["sigma"], rtol=1e-10, atol=1e-16)
    assert np.allclose(st[24:40].reshape(4, 4)[:3, :3], a["chol"], rtol=1e-10, atol=1e-16)
    assert np.allclose(w.cpu().numpy(), a["w"], rtol=1e-11, atol=0)
    h.close()


@pytest.mark.parametrize("B", [1, 3, 17, 1024, 4097])
def test_resample_bit_exact(B):
    rng = np.random.default_rng(B + 5)
    w = rng.uniform(0, 1, B) ** 4
    w[rng.integers(0, B)] = 1.0
    if B > 3:
        w[rng.integers(0, B, size=B // 4)] = 0.0
        w[0] = 1.0
    u = synthetic.uniforms(2, synthetic.RESAMPLE, B, B)
    ref = tm.resample(w, u)
    h = _h(B)
    idx, counts = g.tmcmc_resample(h, torch.tensor(w, device=DEV), torch.tensor(u, device=DEV))
    torch.cuda.synchronize()
    assert np.array_equal(idx.cpu().numpy(), ref)
    assert np.array_equal(counts.cpu().numpy(), np.bincount(ref, minlength=B))
    h.close()


# a small swimmer inverse problem: theta = (alpha, log10 K_C, a)
BASE = sw.SwimmerParams(n=12, dt=2e-4, steps=5000, obs_every=250, alpha=1.0, amp=0.1)
LO = np.array([0.0, -1.0, 0.05])
HI = np.array([10.0, 1.0, 0.2])
TRUTH = (1.0, 0.0, 0.1)


def _problem():
    obs, _, _, st = sw.run_c_batch([BASE.with_theta(TRUTH)])
    xi = obs[0]
    sigma = sw.noise_sigma(xi, 0.05)
    D = xi + sigma * synthetic.normals(1234, synthetic.NOISE, 0, xi.size).reshape(xi.shape)
    return D, sigma


def _gpu_run(B, seed, precision, D, sigma):
    cfg = g.SwimmerConfig(n_max=BASE.n, b_max=B, length=BASE.length, dt=BASE.dt, steps=BASE.steps,
                          obs_every=BASE.obs_every, precision=precision)
    h = g.swimmer_init(cfg)
    th0 = torch.tensor(synthetic.prior_samples(seed, LO, HI, B), device=DEV)
    log = []
    st = g.tmcmc_run(h, th0, torch.tensor(D, device=DEV), sigma, LO, HI,
                     lambda j: synthetic.stage_randoms(seed, j, B, 3), log=log)
    torch.cuda.synchronize()
    out = st.theta.cpu().numpy(), st.loglik.cpu().numpy(), log
    h.close()
    return out


def test_tmcmc_fp64_matches_oracle_sample_by_sample():
    B, seed = 96, 42
    D, sigma = _problem()
    th_g, ll_g, log_g = _gpu_run(B, seed, g.FP64, D, sigma)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count())) as pool:
        fn = lambda th: sw.batch_log_likelihood(BASE, th, D, sigma, pool=pool, chunk=4)
        th_o, ll_o, log_o = tm.run(synthetic.prior_samples(seed, LO, HI, B), fn, LO, HI, seed,
                                   randoms=lambda j: synthetic.stage_randoms(seed, j, B, 3))
    assert [s["q"] for s in log_g] == pytest.approx(log_o.q, rel=1e-9)
    assert [s["unique"] for s in log_g] == log_o.unique
    # model evidence log p(D|M) = sum_j log S_j (Sec. 3.2), accumulated in the state
    assert log_g[-1]["log_evidence"] == pytest.approx(sum(log_o.log_s), rel=1e-9)
    assert np.allclose(th_g, th_o, rtol=1e-8, atol=1e-10)
    assert np.allclose(ll_g, ll_o, rtol=1e-8, atol=1e-8)


def _moment_gaps(th32, th64, B):
    """Gaps of the FP32 run's posterior means and sds from the FP64 run's, and the tolerance
    each meets.  2 % is relative to the FP64 value: for a mean, 2 % of |mean| or of the
    posterior sd when the mean lies closer to zero than one sd (a relative error of a mean
    near zero means nothing).  The Monte-Carlo tolerance is two standard errors of the
    difference of two runs that have decoupled (a flipped Metropolis decision makes the rest
    of the two chains independent): TMCMC holds the weights' COV at 1, an effective sample
    size of B / 2, so SE(mean) = sqrt(2) sd / sqrt(B / 2) and SE(sd) = sd / sqrt(B / 2)."""
    m64, s64, m32, s32 = th64.mean(0), th64.std(0), th32.mean(0), th32.std(0)
    ess = B / 2.0
    tol_m = np.maximum(0.02 * np.maximum(np.abs(m64), s64), 2 * np.sqrt(2.0) * s64 / np.sqrt(ess))
    tol_s = np.maximum(0.02 * s64, 2 * s64 / np.sqrt(ess))
    return np.abs(m32 - m64), tol_m, np.abs(s32 - s64), tol_s, 0.02 * np.maximum(np.abs(m64), s64), 0.02 * s64


def test_tmcmc_fp32_posterior_within_2pct_of_fp64_at_the_workload_size():
    """The precision form of the FP32 kernel against FP64, on the TMCMC workload's swimmer
    (N = 128, dt = 1e-4/64, 1024 samples per stage, the workload's prior) over a shortened
    horizon (2000 Euler steps, head observed every 100, noise 5 % of the head's mean
    displacement so that the run takes several stages).  Sec. 3.2, Algorithm 1.

    (1) The target posteriors: the FP64 model's posterior moments follow from the FP32 run's
    final samples by reweighting them with exp(l64 - l32), the two estimates sharing their
    Monte-Carlo error; they are within 2 % of the FP32 moments.  Since the weights lie within
    exp(+-2 eps), eps = max|l32 - l64|, the means can move by at most about 2 eps times the
    posterior sd, which the test also checks.  (2) Two TMCMC runs sharing every random number, one per kernel:
    their moments are compared at 2 % or, where a decision flipped and the chains decoupled,
    at the Monte-Carlo tolerance of two decoupled runs (``_moment_gaps``)."""
    p = sw.SwimmerParams(n=128, dt=1e-4 / 64, steps=2000, obs_every=100, k_t=1e3)
    B, seed = 1024, 610
    obs, _, _, _ = sw.run_c_batch([p.with_theta(TRUTH)])
    xi = obs[0]
    sigma = 0.05 * float(np.mean(np.abs(xi - [p.length, 0.0])))
    D = torch.tensor(xi + sigma * synthetic.normals(1236, synthetic.NOISE, 0, xi.size).reshape(xi.shape), device=DEV)
    th0 = torch.tensor(synthetic.prior_samples(seed, LO, HI, B), device=DEV)
    out = {}
    handles = {}
    for name, prec in (("fp64", g.FP64), ("fp32", g.FP32C)):
        h = g.swimmer_init(g.SwimmerConfig(n_max=p.n, b_max=B, length=p.length, dt=p.dt, k_t=p.k_t, steps=p.steps,
                                           obs_every=p.obs_every, precision=prec))
        log = []
        st = g.tmcmc_run(h, th0, D, sigma, LO, HI, lambda j: synthetic.stage_randoms(seed, j, B, 3), log=log)
        torch.cuda.synchronize()
        out[name] = (st.theta.clone(), st.loglik.clone(), log)
        handles[name] = h
    th32, ll32, log32 = out["fp32"]
    th64, _, log64 = out["fp64"]
    assert log32[-1]["q"] == 1.0 and log64[-1]["q"] == 1.0 and len(log64) >= 3
    # (1) the FP64 model's log-likelihood at the FP32 run's final samples
    ll64_at32, st64 = g.loglik_batch(handles["fp64"], th32, D, sigma)
    torch.cuda.synchronize()
    for h in handles.values():
        h.close()
    a, b = ll32.cpu().numpy(), ll64_at32.cpu().numpy()
    assert np.all(st64.cpu().numpy() == 0)
    eps = np.max(np.abs(a - b))
    assert eps < 0.05, eps  # a few 1e-3 nats here; runs near the stability edge reach 0.03
    t = th32.cpu().numpy()
    w = np.exp(b - a)
    w /= w.sum()
    m_rw = w @ t
    s_rw = np.sqrt(w @ (t - m_rw) ** 2)
    m32, s32 = t.mean(0), t.std(0)
    assert np.all(np.abs(m_rw - m32) <= 0.02 * np.maximum(np.abs(m32), s32)), (m_rw, m32)
    assert np.all(np.abs(s_rw - s32) <= 0.02 * s32), (s_rw, s32)
    # the reweighting bound itself: |w_k B - 1| <= exp(2 eps) - 1, so the means move by at most
    # about 2 eps times the mean absolute deviation, which is at most the sd
    assert np.all(np.abs(m_rw - m32) <= 2.1 * eps * s32 + 1e-15)
    # (2) the two coupled runs
    dm, tol_m, ds, tol_s, pct_m, pct_s = _moment_gaps(t, th64.cpu().numpy(), B)
    assert np.all(dm <= tol_m), (dm, tol_m)
    assert np.all(ds <= tol_s), (ds, tol_s)
    same = [s["n_accept"] for s in log32] == [s["n_accept"] for s in log64]
    if same:  # every decision agreed: the moments agree far inside 2 %
        assert np.all(dm <= pct_m) and np.all(ds <= pct_s), (dm, pct_m, ds, pct_s)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_stage_sums_to_the_whole_stage(world):
    from paper_1910_12007_gb300 import ranks

    B, seed = 256, 3
    D, sigma = _problem()
    cfg = g.SwimmerConfig(n_max=BASE.n, b_max=B, length=BASE.length, dt=BASE.dt, steps=BASE.steps,
                          obs_every=BASE.obs_every, precision=g.FP32C)
    h = g.swimmer_init(cfg)
    obs = torch.tensor(D, device=DEV)
    th0 = torch.tensor(synthetic.prior_samples(seed, LO, HI, B), device=DEV)
    ll0, _ = g.loglik_batch(h, th0, obs, sigma)
    u_res, u_acc, z = synthetic.stage_randoms(seed, 0, B, 3)
    U = torch.tensor(np.concatenate([u_res[None], u_acc]), device=DEV)
    Z = torch.tensor(z, device=DEV)

    def fresh():
        return g.TmcmcState(th0.clone(), ll0.clone(), obs, sigma, LO, HI)

    full = fresh()
    g.tmcmc_stage(h, full, U, Z)
    parts = []
    for r in range(world):
        s = fresh()
        g.tmcmc_stage(h, s, U, Z, rank=r, world=world)
        parts.append(s)
    torch.cuda.synchronize()
    # which rows each rank owns: the documented rule on the stage's resample counts
    w, _ = g.tmcmc_analyze(h, th0, ll0, 0.0)
    _, counts = g.tmcmc_resample(h, w, U[0].contiguous())
    counts = counts.cpu().numpy()
    owner = ranks.chain_owner(counts, world)
    row_owner = np.concatenate([[owner[k]] * int(counts[k]) for k in range(B) if counts[k] > 0])
    th_full, ll_full = full.theta.cpu().numpy(), full.loglik.cpu().numpy()
    tot_th = np.zeros_like(th_full)
    tot_ll = np.zeros_like(ll_full)
    for r, s in enumerate(parts):
        th, ll = s.theta.cpu().numpy(), s.loglik.cpu().numpy()
        mine = row_owner == r
        assert mine.any()
        assert np.array_equal(th[mine], th_full[mine]) and np.array_equal(ll[mine], ll_full[mine])
        assert not th[~mine].any() and not ll[~mine].any()
        assert s.q == full.q and s.c.max_chain == full.c.max_chain
        tot_th += th
        tot_ll += ll
    assert np.array_equal(tot_th, th_full) and np.array_equal(tot_ll, ll_full)
    assert sum(s.c.n_accept for s in parts) == full.c.n_accept
    assert sum(s.c.n_exact_path for s in parts) == full.c.n_exact_path
    # the blocks are balanced by chain length: each within one chain of B / world rows
    loads = np.bincount(row_owner, minlength=world)
    assert np.all(np.abs(loads - B / world) <= counts.max())
    h.close()


def test_tmcmc_with_the_noise_level_as_a_fourth_unknown():
    # sigma/beta inferred (Sec. 3.1): theta = (alpha, log10 K_C, a, s), the sample's noise is
    # s * beta.  FP64 path sample by sample against the oracle, whose likelihood reads the
    # fourth column the same way
    B, seed = 96, 43
    D, sigma = _problem()
    beta = sigma / 0.05
    lo4, hi4 = np.append(LO, 0.01), np.append(HI, 0.2)
    cfg = g.SwimmerConfig(n_max=BASE.n, b_max=B, length=BASE.length, dt=BASE.dt, steps=BASE.steps,
                          obs_every=BASE.obs_every, precision=g.FP64, n_params=4)
    h = g.swimmer_init(cfg)
    th0 = torch.tensor(synthetic.prior_samples(seed, lo4, hi4, B), device=DEV)
    log_g = []
    st = g.tmcmc_run(h, th0, torch.tensor(D, device=DEV), beta, lo4, hi4,
                     lambda j: synthetic.stage_randoms(seed, j, B, 4), log=log_g)
    torch.cuda.synchronize()
    th_g, ll_g = st.theta.cpu().numpy(), st.loglik.cpu().numpy()
    h.close()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count())) as pool:
        fn = lambda th: sw.batch_log_likelihood(BASE, th, D, beta, pool=pool, chunk=4)
        th_o, ll_o, log_o = tm.run(synthetic.prior_samples(seed, lo4, hi4, B), fn, lo4, hi4, seed,
                                   randoms=lambda j: synthetic.stage_randoms(seed, j, B, 4))
    assert th_g.shape == (B, 4)
    assert [s["q"] for s in log_g] == pytest.approx(log_o.q, rel=1e-9)
    assert np.allclose(th_g, th_o, rtol=1e-8, atol=1e-10)
    assert np.allclose(ll_g, ll_o, rtol=1e-8, atol=1e-8)
    # the noise level the data were made with (5 %) lies inside the posterior's bulk
    s = th_g[:, 3]
    assert np.quantile(s, 0.02) < 0.05 < np.quantile(s, 0.98)


def test_tmcmc_stage_at_the_workload_size_matches_oracle():
    """Two stages at the TMCMC workload's size (1024 samples, N = 128, dt = 1e-4/64, the
    workload's prior box), FP64 kernel against the oracle sample by sample.  The run is 200 Euler steps with the head observed every 10,
    and the noise is 5 % of the head's mean displacement, so the stage has informative
    weights and chains of several steps.  At this batch size the stage pre-fetches chain
    steps in decision trees sized by the GPU's resident capacity, which the small problems
    above never reach."""
    p = sw.SwimmerParams(n=128, dt=1e-4 / 64, steps=200, obs_every=10, k_t=1e3)
    B, seed, P = 1024, 45, 3
    obs, _, _, st = sw.run_c_batch([p.with_theta(TRUTH)])
    xi = obs[0]
    sigma = 0.05 * float(np.mean(np.abs(xi - [p.length, 0.0])))
    D = xi + sigma * synthetic.normals(1235, synthetic.NOISE, 0, xi.size).reshape(xi.shape)
    th0 = synthetic.prior_samples(seed, LO, HI, B)
    cfg = g.SwimmerConfig(n_max=p.n, b_max=B, length=p.length, dt=p.dt, k_t=p.k_t, steps=p.steps,
                          obs_every=p.obs_every, precision=g.FP64)
    h = g.swimmer_init(cfg)
    obs_d = torch.tensor(D, device=DEV)
    ll0, _ = g.loglik_batch(h, torch.tensor(th0, device=DEV), obs_d, sigma)
    stg = g.TmcmcState(torch.tensor(th0, device=DEV), ll0, obs_d, sigma, LO, HI)
    log_g = []
    for j in range(2):
        u_res, u_acc, z = synthetic.stage_randoms(seed, j, B, P)
        U = torch.tensor(np.concatenate([u_res[None], u_acc]), device=DEV)
        log_g.append(g.tmcmc_stage(h, stg, U, torch.tensor(z, device=DEV)))
    torch.cuda.synchronize()
    th_g, ll_g = stg.theta.cpu().numpy(), stg.loglik.cpu().numpy()
    h.close()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count())) as pool:
        fn = lambda th: sw.batch_log_likelihood(p, th, D, sigma, pool=pool, chunk=8)
        th_o, ll_o, log_o = tm.run(th0, fn, LO, HI, seed, max_stages=2,
                                   randoms=lambda j: synthetic.stage_randoms(seed, j, B, P))
    assert [s["q"] for s in log_g] == pytest.approx(log_o.q, rel=1e-9)
    assert [s["unique"] for s in log_g] == log_o.unique
    assert [s["n_exact_path"] for s in log_g] == log_o.n_exact
    assert max(s["max_chain"] for s in log_g) >= 4
    assert np.allclose(th_g, th_o, rtol=1e-8, atol=1e-10)
    fin = np.isfinite(ll_o)
    assert np.array_equal(fin, np.isfinite(ll_g))
    assert np.allclose(ll_g[fin], ll_o[fin], rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("precision", [g.FP32C, g.FP64])
def test_stage_async_captured_in_a_graph_replays_the_eager_stage(precision):
    """tmcmc_stage_async enqueues a whole stage (Sec. 3.2, Algorithm 1) with no host
    synchronization: the Metropolis chains' pre-fetch rounds run as a loop whose condition the
    device sets.  Captured in a CUDA graph, every replay from the same inputs reproduces the
    eager stage bit for bit, as does the host-driven loop used under profiling."""
    from paper_1910_12007_gb300 import api

    B, seed = 256, 46
    D, sigma = _problem()
    cfg = g.SwimmerConfig(n_max=BASE.n, b_max=B, length=BASE.length, dt=BASE.dt, steps=BASE.steps,
                          obs_every=BASE.obs_every, precision=precision)
    h = g.swimmer_init(cfg)
    obs = torch.tensor(D, device=DEV)
    th0 = torch.tensor(synthetic.prior_samples(seed, LO, HI, B), device=DEV)
    ll0, _ = g.loglik_batch(h, th0, obs, sigma)
    u_res, u_acc, z = synthetic.stage_randoms(seed, 0, B, 3)
    U = torch.tensor(np.concatenate([u_res[None], u_acc]), device=DEV)
    Z = torch.tensor(z, device=DEV)
    # the synchronous stage (graph of its own) and the same stage with host-driven rounds
    e = g.TmcmcState(th0.clone(), ll0.clone(), obs, sigma, LO, HI)
    g.tmcmc_stage(h, e, U, Z)
    p = g.TmcmcState(th0.clone(), ll0.clone(), obs, sigma, LO, HI)
    g.swimmer_profile(h, 1)
    g.tmcmc_stage(h, p, U, Z)
    g.swimmer_profile(h, 0)
    torch.cuda.synchronize()
    assert torch.equal(p.theta, e.theta) and torch.equal(p.loglik, e.loglik)
    assert e.c.max_chain >= 2 and 0 < e.q < 1
    # asynchronous: the exponent and the summary stay on the device
    s = g.TmcmcState(th0.clone(), ll0.clone(), obs, sigma, LO, HI)
    q = torch.zeros(1, dtype=torch.float64, device=DEV)
    summ = torch.zeros(api.STAGE_SUMMARY, dtype=torch.float64, device=DEV)
    g.tmcmc_stage_async(h, s, U, Z, q, summ)
    torch.cuda.synchronize()
    assert torch.equal(s.theta, e.theta) and torch.equal(s.loglik, e.loglik)

    def check_summary():
        r = summ.cpu().numpy()
        assert r[api.STAGE_STATUS] == 0 and r[api.STAGE_Q_IN] == 0.0
        assert r[api.STAGE_Q] == e.q == q.item()
        assert r[api.STAGE_LOG_S] == e.c.log_s
        assert int(r[api.STAGE_UNIQUE]) == e.c.unique and int(r[api.STAGE_MAX_CHAIN]) == e.c.max_chain
        assert int(r[api.STAGE_ACCEPT]) == e.c.n_accept and int(r[api.STAGE_EXACT_PATH]) == e.c.n_exact_path

    check_summary()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        g.tmcmc_stage_async(h, s, U, Z, q, summ)
    for _ in range(2):
        s.theta.copy_(th0)
        s.loglik.copy_(ll0)
        q.zero_()
        summ.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(s.theta, e.theta) and torch.equal(s.loglik, e.loglik)
        check_summary()
    del graph
    h.close()


def test_stage_rounds_at_the_workload_size_same_in_graph_and_host_loop():
    """At the TMCMC workload's size (1024 samples, N = 128, FP32, autotuned launch shapes) the
    pre-fetch rounds launch their forward runs with the shape and grid of the rows that run:
    a switch node selects the branch on the device inside the stage graph, and the
    host-driven loop (profiling) reads the same count.  Both must give the same stage bit for
    bit, every round's recorded rows must be positive and no more than the rows a round can
    hold, and together they cover every chain step (Algorithm 1: one exact run per step)."""
    p = sw.SwimmerParams(n=128, dt=1e-4 / 64, steps=400, obs_every=10, k_t=1e3)
    B, seed, P = 1024, 47, 3
    obs, _, _, _ = sw.run_c_batch([p.with_theta(TRUTH)])
    xi = obs[0]
    sigma = 0.05 * float(np.mean(np.abs(xi - [p.length, 0.0])))
    D = xi + sigma * synthetic.normals(1236, synthetic.NOISE, 0, xi.size).reshape(xi.shape)
    cfg = g.SwimmerConfig(n_max=p.n, b_max=B, length=p.length, dt=p.dt, k_t=p.k_t, steps=p.steps,
                          obs_every=p.obs_every, precision=g.FP32C)
    h = g.swimmer_init(cfg)
    th0 = torch.tensor(synthetic.prior_samples(seed, LO, HI, B), device=DEV)
    g.swimmer_autotune(h, steps=200, theta=th0)
    obs_d = torch.tensor(D, device=DEV)
    ll0, _ = g.loglik_batch(h, th0, obs_d, sigma)
    states = {}
    for mode in ("graph", "host"):
        st = g.TmcmcState(th0.clone(), ll0.clone(), obs_d, sigma, LO, HI)
        for j in range(3):
            u_res, u_acc, z = synthetic.stage_randoms(seed, j, B, P)
            U = torch.tensor(np.concatenate([u_res[None], u_acc]), device=DEV)
            if mode == "host":
                g.swimmer_profile(h, 1)
            s = g.tmcmc_stage(h, st, U, torch.tensor(z, device=DEV))
            if mode == "host":
                rounds = g.swimmer_profile_launches(h)
                g.swimmer_profile(h, 0)
                runs = [n for _, n in rounds]
                assert len(runs) >= 2 and all(0 < n <= B for n in runs), runs
                # every chain step ran once on its realized path; speculative runs add to that
                assert sum(runs) >= s["n_exact_path"]
        torch.cuda.synchronize()
        states[mode] = (st.theta.clone(), st.loglik.clone(), st.q)
    h.close()
    assert torch.equal(states["graph"][0], states["host"][0])
    assert torch.equal(states["graph"][1], states["host"][1])
    assert states["graph"][2] == states["host"][2]
