"""Transitional Markov chain Monte Carlo, FP64 (oracle; test infrastructure only).

Follows Sec. 3.2 and Algorithm 1:
* intermediate targets f_j ~ p(D|theta)^{q_j} pi(theta), 0 = q_0 < ... < q_lambda = 1;
* analyze: choose q_{j+1} so that the coefficient of variation of the plausibility
  weights w_k = p(D|theta_k)^{q_{j+1} - q_j} equals the tolerance (1.0); S_j = mean(w),
  normalized weights w_bar = w / sum(w), sample mean mu_j and scaled covariance
  Sigma_j = b^2 sum_k w_bar_k (theta_k - mu_j)(theta_k - mu_j)^T, b = 0.2;
* resample: theta_hat_{j+1,l} = theta_{j,k} with probability w_bar_k; n_{j+1,k} copies;
* each unique sample seeds a Metropolis chain of length n_{j+1,k} with Gaussian
  proposal N(theta, Sigma_j) and target f_{j+1};
* stop after the stage run at q = 1.

Readings where the paper is loose (the same readings the CUDA path takes):
* "covariance of the weights ... smaller than a tolerance, often 1.0" -> the coefficient of
  variation (population standard deviation / mean) equals 1.0; bisection on
  dq in (0, 1 - q_j], 200 halvings or until the bracket is below 1e-15; if the COV at
  dq = 1 - q_j is <= 1, q_{j+1} = 1.
* "sampled uniformly at random ... with probability w_bar" -> multinomial by w_bar, by
  the inverse CDF of a 64-bit fixed-point prefix sum: W_k = floor(w_k 2^40) with
  w_k = exp(dq (l_k - l_max)) in [0, 1], C = inclusive prefix of W, target
  t = min(floor(u C_B), C_B - 1), index = min{i : C_i > t}.
* Metropolis target f_j -> f_{j+1} (the chains run after q_{j+1} is chosen).
* Uniform box prior: a proposal outside the box is rejected without a likelihood call.
* Chain c (for the c-th unique index in ascending order) writes its n_c outputs to
  positions off_c .. off_c + n_c - 1 (off = exclusive prefix of the counts); its step s
  uses normals z[off_c + s] and uniforms u_acc[off_c + s].
* Diverged forward runs have log-likelihood -inf, i.e. weight 0.

Delayed acceptance (not in the paper): a cheap surrogate l~ screens each proposal first;
step 1 accepts with min(1, exp(q (l~' - l~))), step 2 with
min(1, exp(q (l' - l) - q (l~' - l~))), the two-stage Metropolis-Hastings rule that keeps
the exact target for a symmetric proposal.  The plain model judges the surrogate: over the
proposals a stage evaluates with both (at least 10, finite l), err = q_{j+1} times the
population standard deviation of l - l~ (a constant offset cancels in the screen's ratio);
the next stage screens only if err <= 1 nat, else it runs plain Metropolis (row 0 of the
acceptance uniforms), still evaluating the surrogate.  A run starts trusting the surrogate.

Pins (tests/test_oracle_tmcmc.py): Gaussian toy posterior mean/variance (closed form);
the COV at the chosen q equals 1; the resample against brute-force inverse-CDF search;
sum of counts = number of samples; final q = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FIXED_BITS = 40
COV_TARGET = 1.0
B_SCALE = 0.2
SURROGATE_ERR_MAX = 1.0    # nats
SURROGATE_MIN_JUDGED = 10


def _weights(loglik, dq):
    l = np.asarray(loglik, dtype=np.float64)
    fin = np.isfinite(l)
    lmax = np.max(l[fin])
    w = np.zeros_like(l)
    w[fin] = np.exp(dq * (l[fin] - lmax))
    return w, lmax


def cov_of_weights(loglik, dq):
    w, _ = _weights(loglik, dq)
    m = np.mean(w)
    return math.sqrt(np.mean((w - m) ** 2)) / m


def solve_dq(loglik, q):
    """Increment dq of the annealing exponent with COV(w) = 1 (bisection)."""
    hi = 1.0 - q
    if cov_of_weights(loglik, hi) <= COV_TARGET:
        return hi
    lo = 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if cov_of_weights(loglik, mid) > COV_TARGET:
            hi = mid
        else:
            lo = mid
        if hi - lo < 1e-15:
            break
    return 0.5 * (lo + hi)


def analyze(theta, loglik, q):
    """Algorithm 1 'Analyze': q_{j+1}, weights, log S_j, mu_j, Sigma_j and its Cholesky factor."""
    theta = np.asarray(theta, dtype=np.float64)
    dq = solve_dq(loglik, q)
    w, lmax = _weights(loglik, dq)
    q_next = 1.0 if q + dq >= 1.0 - 1e-15 else q + dq
    wbar = w / np.sum(w)
    log_s = dq * lmax + math.log(np.mean(w))
    mu = wbar @ theta
    dev = theta - mu
    sigma = B_SCALE ** 2 * (dev * wbar[:, None]).T @ dev
    chol = np.linalg.cholesky(sigma)
    return dict(dq=dq, q_next=q_next, w=w, wbar=wbar, log_s=log_s, mu=mu, sigma=sigma, chol=chol)


def resample(w, u):
    """Multinomial resampling by inverse CDF on the 64-bit fixed-point prefix sum."""
    W = np.floor(np.asarray(w, dtype=np.float64) * 2.0 ** FIXED_BITS).astype(np.int64)
    C = np.cumsum(W)
    total = int(C[-1])
    t = np.minimum(np.floor(np.asarray(u) * float(total)).astype(np.int64), total - 1)
    return np.searchsorted(C, t, side="right").astype(np.int64)


def chains(idx, n_samples):
    """Unique resampled indices (ascending), their counts and output offsets."""
    counts = np.bincount(idx, minlength=n_samples)
    uniq = np.nonzero(counts)[0]
    n_c = counts[uniq]
    off = np.concatenate([[0], np.cumsum(n_c)[:-1]])
    return uniq, n_c, off


def in_support(theta, lo, hi):
    return bool(np.all(theta >= lo) and np.all(theta <= hi))


def metropolis(theta, loglik, idx, chol, q_next, z, u_acc, lo, hi, loglik_fn,
               surrogate_fn=None, surr=None, trust=True):
    """Run the Metropolis chains of one stage.

    loglik_fn(thetas[m, P]) -> logliks[m] evaluates the exact model on a batch.
    With ``surrogate_fn`` (delayed acceptance) ``surr`` holds the surrogate logliks of the
    current samples; ``trust`` False runs plain Metropolis while still evaluating it.  Returns
    new theta, loglik (and surrogate logliks), counters and the values l - l~ of the proposals
    evaluated with both."""
    B, P = theta.shape
    uniq, n_c, off = chains(idx, B)
    out_t = np.zeros_like(theta)
    out_l = np.zeros(B)
    out_s = np.zeros(B) if surrogate_fn is not None else None
    cur_t = theta[uniq].copy()
    cur_l = loglik[uniq].copy()
    cur_s = surr[uniq].copy() if surrogate_fn is not None else None
    n_exact = 0
    n_accept = 0
    n_pass1 = 0
    judged = []
    for s in range(int(n_c.max())):
        act = np.nonzero(n_c > s)[0]
        pos = off[act] + s
        prop = cur_t[act] + z[pos] @ chol.T
        ok = np.array([in_support(t, lo, hi) for t in prop])
        cand = act[ok]
        cpos = pos[ok]
        cprop = prop[ok]
        acc = np.zeros(len(act), dtype=bool)
        if len(cand):
            if surrogate_fn is None:
                lp = loglik_fn(cprop)
                n_exact += len(cand)
                a = np.log(u_acc[0, cpos]) < q_next * (lp - cur_l[cand])
                sel = cand[a]
                cur_t[sel] = cprop[a]
                cur_l[sel] = lp[a]
            elif not trust:  # plain Metropolis, the surrogate still evaluated and judged
                sp = surrogate_fn(cprop)
                lp = loglik_fn(cprop)
                n_exact += len(cand)
                fin = np.isfinite(lp)
                judged.extend((lp - sp)[fin])
                a = np.log(u_acc[0, cpos]) < q_next * (lp - cur_l[cand])
                sel = cand[a]
                cur_t[sel] = cprop[a]
                cur_l[sel] = lp[a]
                cur_s[sel] = sp[a]
            else:
                sp = surrogate_fn(cprop)
                a1 = np.log(u_acc[0, cpos]) < q_next * (sp - cur_s[cand])
                n_pass1 += int(np.sum(a1))
                c2 = cand[a1]
                if len(c2):
                    lp = loglik_fn(cprop[a1])
                    n_exact += len(c2)
                    judged.extend((lp - sp[a1])[np.isfinite(lp)])
                    a2 = np.log(u_acc[1, cpos[a1]]) < q_next * (lp - cur_l[c2]) - q_next * (sp[a1] - cur_s[c2])
                    sel = c2[a2]
                    cur_t[sel] = cprop[a1][a2]
                    cur_l[sel] = lp[a2]
                    cur_s[sel] = sp[a1][a2]
                    a = np.zeros(len(cand), dtype=bool)
                    a[np.nonzero(a1)[0][a2]] = True
                else:
                    a = np.zeros(len(cand), dtype=bool)
            acc[np.nonzero(ok)[0]] = a
        n_accept += int(np.sum(acc))
        out_t[pos] = cur_t[act]
        out_l[pos] = cur_l[act]
        if out_s is not None:
            out_s[pos] = cur_s[act]
    return dict(theta=out_t, loglik=out_l, surr=out_s, n_exact=n_exact, n_accept=n_accept,
                n_pass1=n_pass1, unique=len(uniq), max_chain=int(n_c.max()), judged=np.array(judged))


@dataclass
class StageLog:
    q: list = field(default_factory=list)
    log_s: list = field(default_factory=list)
    accept: list = field(default_factory=list)
    unique: list = field(default_factory=list)
    n_exact: list = field(default_factory=list)
    surrogate_used: list = field(default_factory=list)
    surrogate_error: list = field(default_factory=list)


def run(theta0, loglik_fn, lo, hi, seed, surrogate_fn=None, max_stages=100, randoms=None):
    """Algorithm 1.  ``randoms(stage) -> (u_res[B], u_acc[2, B], z[B, P])``."""
    theta = np.array(theta0, dtype=np.float64)
    B, P = theta.shape
    loglik = loglik_fn(theta)
    surr = surrogate_fn(theta) if surrogate_fn is not None else None
    q = 0.0
    log = StageLog()
    trust = True
    for j in range(max_stages):
        a = analyze(theta, loglik, q)
        u_res, u_acc, z = randoms(j)
        idx = resample(a["w"], u_res)
        m = metropolis(theta, loglik, idx, a["chol"], a["q_next"], z, u_acc, lo, hi, loglik_fn,
                       surrogate_fn, surr, trust)
        theta, loglik, surr = m["theta"], m["loglik"], m["surr"]
        q = a["q_next"]
        if surrogate_fn is not None:
            log.surrogate_used.append(trust)
            d = m["judged"]
            err = q * float(np.std(d)) if len(d) >= SURROGATE_MIN_JUDGED else float("nan")
            log.surrogate_error.append(err)
            if len(d) >= SURROGATE_MIN_JUDGED:
                trust = err <= SURROGATE_ERR_MAX
        log.q.append(q)
        log.log_s.append(a["log_s"])
        log.accept.append(m["n_accept"] / B)
        log.unique.append(m["unique"])
        log.n_exact.append(m["n_exact"])
        if q >= 1.0:
            break
    return theta, loglik, log
