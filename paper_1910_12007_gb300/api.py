"""Thin Python binding over the C ABI (include/swimmer.h): argument marshalling only.

Device memory comes from PyTorch tensors; every step of the computation runs in the
CUDA kernels of libswimmer.so.  Function names follow the C entry points.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, fields

import torch

from ._lib import SwimmerConfigC, TmcmcStateC, check, lib

FP64 = 0
FP32C = 1
SHAPE_WIDE = 0x10000  # launch-shape flag (FP32C): two target blocks per pair unit
SHAPE_QUAD = 0x20000  # launch-shape flag (FP32C): four target blocks per pair unit


OBS_HEAD_POINT, OBS_HEAD_VELOCITY, OBS_PAIR_DISTANCES = 0, 1, 2


@dataclass
class SwimmerConfig:
    """Mirror of ``swimmer_config`` (physical and numerical parameters, Table Tab:param)."""

    n_max: int = 64
    b_max: int = 1
    length: float = 1.0
    ds_fixed: float = 0.0
    mu: float = 1.0
    delta_over_ds: float = 1.5
    dt: float = 1.25e-5
    k_t: float = 1e3
    eta: float = 2 * math.pi
    omega: float = 2 * math.pi
    steps: int = 80000
    obs_every: int = 800
    precision: int = FP32C
    # full sperm model (head and neck); n_head = 0 is the flagellum alone
    n_head: int = 0
    head_radius_over_ds: float = 0.0
    neck_gap_over_ds: float = 0.0
    k_head_tens: float = 1e4
    k_head_c: float = 0.8
    k_neck_tens: float = 500.0
    k_neck_ang: float = 1e4
    obs_kind: int = 0  # OBS_HEAD_POINT, OBS_HEAD_VELOCITY or OBS_PAIR_DISTANCES
    # two swimmers per sample; noise ratio of the second observed component
    n_swimmers: int = 1
    swimmer_distance: float = 2.0
    sigma_ratio: float = 0.0
    # unknowns per sample: 3, or 4 with the noise level (sigma = theta[3] * sigma)
    n_params: int = 3

    def to_c(self):
        return SwimmerConfigC(**{f.name: getattr(self, f.name) for f in fields(self)})

    @property
    def n_obs(self):
        return self.steps // self.obs_every


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA tensor of dtype {dtype}")
    return t


class Handle:
    """Owns a ``swimmer_handle`` (device workspaces for b_max samples)."""

    def __init__(self, cfg: SwimmerConfig):
        self.cfg = cfg
        self._c = cfg.to_c()
        h = ctypes.c_void_p()
        check(lib().swimmer_init(ctypes.byref(self._c), ctypes.byref(h)))
        self.ptr = h

    def close(self):
        if self.ptr:
            lib().swimmer_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def swimmer_init(cfg: SwimmerConfig) -> Handle:
    return Handle(cfg)


def swimmer_destroy(h: Handle):
    h.close()


def swimmer_kernel_eval(h: Handle, alpha, delta, r_max, r: torch.Tensor, precision=FP64, stream=None):
    """g1 = B'', g2 = (r B'' - B')/r^3 at distances r (CUDA FP64 tensor) through the tables."""
    _dev(r, torch.float64)
    g1 = torch.empty_like(r)
    g2 = torch.empty_like(r)
    check(lib().swimmer_kernel_eval(h.ptr, float(alpha), float(delta), float(r_max), r.numel(),
                                    _ptr(r), _ptr(g1), _ptr(g2), int(precision), _stream(stream)))
    return g1, g2


def forward_batch(h: Handle, theta: torch.Tensor, n_pts=None, want_traj=True, stream=None, out=None):
    """Forward model of B samples: theta [B, 3] (alpha, log10 K_C, a) FP64 on the device.
    Returns (head_traj [B, n_obs, 2] or None, mean_speed [B], status [B])."""
    _dev(theta, torch.float64)
    B = theta.shape[0]
    if n_pts is not None:
        _dev(n_pts, torch.int32)
    dev = theta.device
    if out is None:
        traj = torch.empty((B, h.cfg.n_obs, 2), dtype=torch.float64, device=dev) if want_traj else None
        speed = torch.empty(B, dtype=torch.float64, device=dev)
        status = torch.empty(B, dtype=torch.int32, device=dev)
    else:
        traj, speed, status = out
    check(lib().forward_batch(h.ptr, B, _ptr(theta), _ptr(n_pts), _ptr(traj), _ptr(speed), _ptr(status),
                              _stream(stream)))
    return traj, speed, status


def forward_batch_state(h: Handle, theta: torch.Tensor, n_pts=None, stream=None):
    """forward_batch plus each run's final state [B, n_max, 4] = (x, y, F_x, F_y) at the end
    of the run (NaN rows past a sample's points).  Returns (head_traj, mean_speed, status,
    state)."""
    _dev(theta, torch.float64)
    B = theta.shape[0]
    dev = theta.device
    traj = torch.empty((B, h.cfg.n_obs, 2), dtype=torch.float64, device=dev)
    speed = torch.empty(B, dtype=torch.float64, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    state = torch.empty((B, h.cfg.n_max, 4), dtype=torch.float64, device=dev)
    if n_pts is not None:
        _dev(n_pts, torch.int32)
    check(lib().forward_batch_state(h.ptr, B, _ptr(theta), _ptr(n_pts), _ptr(traj), _ptr(speed), _ptr(status),
                                    _ptr(state), _stream(stream)))
    return traj, speed, status, state


def swimmer_flow_field(h: Handle, alpha, delta, r_max, state: torch.Tensor, grid: torch.Tensor, stream=None):
    """Velocity [G, 2] and pressure [G] at the target points grid [G, 2] (device FP64) from
    the points of state [n, 4] = (x, y, F_x, F_y) (device FP64)."""
    _dev(state, torch.float64)
    _dev(grid, torch.float64)
    G = grid.shape[0]
    vel = torch.empty((G, 2), dtype=torch.float64, device=grid.device)
    pres = torch.empty(G, dtype=torch.float64, device=grid.device)
    check(lib().swimmer_flow_field(h.ptr, float(alpha), float(delta), float(r_max), int(state.shape[0]),
                                   _ptr(state), int(G), _ptr(grid), _ptr(vel), _ptr(pres), _stream(stream)))
    return vel, pres


def loglik_batch(h: Handle, theta, obs, sigma, n_pts=None, stream=None, out=None):
    """Gaussian log-likelihood of B samples against observations obs [n_obs, 2]."""
    _dev(theta, torch.float64)
    _dev(obs, torch.float64)
    B = theta.shape[0]
    if n_pts is not None:
        _dev(n_pts, torch.int32)
    if out is None:
        ll = torch.empty(B, dtype=torch.float64, device=theta.device)
        status = torch.empty(B, dtype=torch.int32, device=theta.device)
    else:
        ll, status = out
    check(lib().loglik_batch(h.ptr, B, _ptr(theta), _ptr(n_pts), _ptr(obs), float(sigma), _ptr(ll),
                             _ptr(status), _stream(stream)))
    return ll, status


# ---------------------------------------------------------------------------------
# TMCMC (Sec. 3.2, Algorithm 1)
# ---------------------------------------------------------------------------------
def tmcmc_analyze(h: Handle, theta, loglik, q, stream=None):
    """Algorithm 1 'Analyze' on the device: returns (w [B], stats [32]) device tensors."""
    _dev(theta, torch.float64)
    _dev(loglik, torch.float64)
    B = loglik.numel()
    w = torch.empty(B, dtype=torch.float64, device=loglik.device)
    stats = torch.zeros(64, dtype=torch.float64, device=loglik.device)
    check(lib().tmcmc_analyze(h.ptr, B, _ptr(theta), _ptr(loglik), float(q), _ptr(w), _ptr(stats), _stream(stream)))
    return w, stats


def tmcmc_resample(h: Handle, w, u, stream=None):
    """Multinomial resampling indices and counts (exact integers) on the device."""
    _dev(w, torch.float64)
    _dev(u, torch.float64)
    B = w.numel()
    idx = torch.empty(B, dtype=torch.int32, device=w.device)
    counts = torch.empty(B, dtype=torch.int32, device=w.device)
    check(lib().tmcmc_resample(h.ptr, B, _ptr(w), _ptr(u), _ptr(idx), _ptr(counts), _stream(stream)))
    return idx, counts


class TmcmcState:
    """Device-resident TMCMC state (theta, loglik) plus the host-side stage summary."""

    def __init__(self, theta, loglik, obs, sigma, prior_lo, prior_hi, surr_loglik=None):
        self.theta = _dev(theta, torch.float64)
        self.loglik = _dev(loglik, torch.float64)
        self.status = torch.zeros(theta.shape[0], dtype=torch.int32, device=theta.device)
        self.obs = _dev(obs, torch.float64)
        self.surr_loglik = surr_loglik
        c = TmcmcStateC()
        c.B = theta.shape[0]
        c.theta = theta.data_ptr()
        c.loglik = loglik.data_ptr()
        c.status = self.status.data_ptr()
        c.n_pts = None
        c.obs = obs.data_ptr()
        c.sigma = float(sigma)
        self.P = theta.shape[1]
        for a in range(self.P):
            c.prior_lo[a] = float(prior_lo[a])
            c.prior_hi[a] = float(prior_hi[a])
        c.q = 0.0
        c.stage = 0
        c.surr_loglik = surr_loglik.data_ptr() if surr_loglik is not None else None
        self.c = c

    @property
    def q(self):
        return self.c.q

    def summary(self):
        c = self.c
        return dict(stage=c.stage, q=c.q, log_s=c.log_s, log_evidence=c.log_evidence, mu=list(c.mu)[:self.P],
                    unique=c.unique,
                    max_chain=c.max_chain, n_exact=c.n_exact, n_screened=c.n_screened, n_accept=c.n_accept,
                    n_exact_path=c.n_exact_path, surrogate_used=c.surrogate_used, surrogate_error=c.surrogate_error)


def tmcmc_tree_template(M, p_accept, depth_cap):
    """The pre-fetch decision tree (host only): list of (parent, depth, is_accept_child,
    accept_child, reject_child) for up to M nodes, root first."""
    buf = (ctypes.c_int * (4 * M))()
    count = ctypes.c_int(0)
    check(lib().tmcmc_tree_template(int(M), float(p_accept), int(depth_cap), buf, ctypes.byref(count)))
    return [(buf[4 * v], buf[4 * v + 1] >> 1, buf[4 * v + 1] & 1, buf[4 * v + 2], buf[4 * v + 3])
            for v in range(count.value)]


def swimmer_pair_units(nb, mode):
    """The FP32 pair sum's work list for nb blocks of 32 points (host only): list of
    (targets, J, d0) per unit of 16 steps: the target blocks (1, 2 or 4), the source block
    and the first step (d0 = 1 marks a diagonal unit, steps 1 .. 16)."""
    buf = (ctypes.c_uint * max(1, nb * nb))()
    count = ctypes.c_int(0)
    check(lib().swimmer_pair_units(int(nb), int(mode), buf, ctypes.byref(count)))
    out = []
    for k in range(count.value):
        u = buf[k]
        kind, code = (u >> 27) & 3, (u >> 25) & 3
        blocks = [u & 31, (u >> 10) & 31, (u >> 15) & 31, (u >> 20) & 31][: (1, 2, 4)[kind]]
        out.append((tuple(blocks), (u >> 5) & 31, 1 if code == 2 else 16 * code))
    return out


def tmcmc_stage(h: Handle, st: TmcmcState, uniforms, normals, use_surrogate=False, stream=None, rank=0, world=1):
    """One TMCMC stage on the device; uniforms [3, B], normals [B, 3] (FP64, device).
    With world > 1 this process runs only rank `rank`'s chains and leaves zeros in the other
    ranks' rows of st.theta / st.loglik (``ranks.assemble_stage`` sums them over ranks)."""
    _dev(uniforms, torch.float64)
    _dev(normals, torch.float64)
    if world == 1:
        check(lib().tmcmc_stage(h.ptr, ctypes.byref(st.c), _ptr(uniforms), _ptr(normals), int(bool(use_surrogate)),
                                _stream(stream)))
    else:
        check(lib().tmcmc_stage_shard(h.ptr, ctypes.byref(st.c), _ptr(uniforms), _ptr(normals),
                                      int(bool(use_surrogate)), int(rank), int(world), _stream(stream)))
    return st.summary()


STAGE_SUMMARY = 32
STAGE_STATUS, STAGE_Q_IN, STAGE_Q, STAGE_LOG_S, STAGE_MU, STAGE_SIGMA = 0, 1, 2, 3, 4, 8
STAGE_UNIQUE, STAGE_MAX_CHAIN, STAGE_ACCEPT, STAGE_SCREENED, STAGE_EXACT, STAGE_EXACT_PATH = 24, 25, 26, 27, 28, 29
STAGE_SURR_USED, STAGE_SURR_ERR = 30, 31


def tmcmc_stage_async(h: Handle, st: TmcmcState, uniforms, normals, q, summary, use_surrogate=False, stream=None,
                      rank=0, world=1):
    """One TMCMC stage enqueued without host synchronization: q (device FP64 [1]) holds the
    annealing exponent in and out, summary (device FP64 [STAGE_SUMMARY]) receives the stage's
    record.  Inside a torch.cuda.graph capture the stage becomes part of the graph."""
    _dev(uniforms, torch.float64)
    _dev(normals, torch.float64)
    _dev(q, torch.float64)
    _dev(summary, torch.float64)
    if q.numel() < 1 or summary.numel() < STAGE_SUMMARY:
        raise ValueError(f"q needs 1 and summary {STAGE_SUMMARY} doubles")
    check(lib().tmcmc_stage_async(h.ptr, ctypes.byref(st.c), _ptr(uniforms), _ptr(normals), int(bool(use_surrogate)),
                                  int(rank), int(world), _ptr(q), _ptr(summary), _stream(stream)))


def tmcmc_run(h: Handle, theta0, obs, sigma, prior_lo, prior_hi, randoms, use_surrogate=False, max_stages=100,
              stream=None, log=None):
    """Algorithm 1 driven from the host: prior samples theta0 [B, 3] (device), observations
    obs [n_obs, 2]; ``randoms(stage) -> (u_res [B], u_acc [2, B], z [B, 3])`` numpy arrays
    (the seeded streams of the ``synthetic`` module).  Returns the final TmcmcState."""
    ll, status = loglik_batch(h, theta0, obs, sigma, stream=stream)
    surr = None
    if use_surrogate:
        surr = surrogate_loglik_batch(h, theta0, obs, sigma, stream=stream)
    st = TmcmcState(theta0.clone(), ll, obs, sigma, prior_lo, prior_hi, surr)
    dev = theta0.device
    for j in range(max_stages):
        u_res, u_acc, z = randoms(j)
        U = torch.tensor(np_stack_uniforms(u_res, u_acc), dtype=torch.float64, device=dev)
        Z = torch.tensor(z, dtype=torch.float64, device=dev)
        s = tmcmc_stage(h, st, U, Z, use_surrogate, stream)
        if log is not None:
            log.append(s)
        if st.q >= 1.0:
            break
    return st


def np_stack_uniforms(u_res, u_acc):
    import numpy as np

    return np.concatenate([np.asarray(u_res)[None, :], np.asarray(u_acc)], axis=0)


# ---------------------------------------------------------------------------------
# learned surrogate (MLP 5 -> 256 -> 256 -> 256 -> 80)
# ---------------------------------------------------------------------------------
MLP_IN, MLP_HIDDEN, MLP_OUT = 5, 256, 80
MLP_NPARAM = 5 * 256 + 256 + 256 * 256 + 256 + 256 * 256 + 256 + 256 * 80 + 80


def mlp_workspace(n, device):
    nbytes = lib().mlp_workspace_bytes(int(n))
    return torch.empty(nbytes // 4 + 1, dtype=torch.float32, device=device)


def mlp_forward(params, x, workspace=None, stream=None):
    _dev(params, torch.float32)
    _dev(x, torch.float32)
    n = x.shape[0]
    y = torch.empty((n, MLP_OUT), dtype=torch.float32, device=x.device)
    ws = workspace if workspace is not None else mlp_workspace(n, x.device)
    check(lib().mlp_forward(n, _ptr(params), _ptr(x), _ptr(y), _ptr(ws), _stream(stream)))
    return y


def mlp_backward(params, x, t, workspace=None, stream=None, grad=None, loss=None):
    _dev(params, torch.float32)
    _dev(x, torch.float32)
    _dev(t, torch.float32)
    n = x.shape[0]
    grad = grad if grad is not None else torch.empty(MLP_NPARAM, dtype=torch.float32, device=x.device)
    loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=x.device)
    ws = workspace if workspace is not None else mlp_workspace(n, x.device)
    check(lib().mlp_backward(n, _ptr(params), _ptr(x), _ptr(t), _ptr(grad), _ptr(loss), _ptr(ws), _stream(stream)))
    return grad, loss


def mlp_adam(params, grad, m, v, step, lr, stream=None):
    check(lib().mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), _stream(stream)))


def swimmer_surrogate_set(h: Handle, params, in_lo, in_hi, out_mean, out_std, obs_stride, log10_kt, omega):
    _dev(params, torch.float32)
    arr = lambda a, n: (ctypes.c_double * n)(*[float(v) for v in a])
    check(lib().swimmer_surrogate_set(h.ptr, _ptr(params), arr(in_lo, 5), arr(in_hi, 5), arr(out_mean, MLP_OUT),
                                      arr(out_std, MLP_OUT), int(obs_stride), float(log10_kt), float(omega)))


def surrogate_loglik_batch(h: Handle, theta, obs, sigma, stream=None):
    _dev(theta, torch.float64)
    _dev(obs, torch.float64)
    ll = torch.empty(theta.shape[0], dtype=torch.float64, device=theta.device)
    check(lib().surrogate_loglik_batch(h.ptr, theta.shape[0], _ptr(theta), _ptr(obs), float(sigma), _ptr(ll),
                                       _stream(stream)))
    return ll


def swimmer_profile(h: Handle, mode):
    """mode 1: start timing forward-kernel launches (CUDA events on their stream) and
    counting kernel launches; mode 2: return (k2_ms, k2_launches, launches,
    executed_pair_evals, useful_pair_evals) and reset; mode 0: stop."""
    out = (ctypes.c_double * 5)()
    check(lib().swimmer_profile(h.ptr, int(mode), out))
    return tuple(out) if mode == 2 else None


def swimmer_profile_launches(h: Handle):
    """(ms, samples) of every forward-kernel launch recorded since profiling started or was
    last reset, oldest first (diagnostic; resets nothing)."""
    count = ctypes.c_int(0)
    check(lib().swimmer_profile_launches(h.ptr, 0, None, None, ctypes.byref(count)))
    n = count.value
    ms = (ctypes.c_double * max(n, 1))()
    samples = (ctypes.c_int * max(n, 1))()
    check(lib().swimmer_profile_launches(h.ptr, n, ms, samples, ctypes.byref(count)))
    return [(ms[i], samples[i]) for i in range(n)]


def swimmer_autotune(h: Handle, steps=200, theta=None):
    """Time the forward kernel's launch shapes per bucket of samples per SM, on `theta`
    ([n, 3] FP64 on the device, representative samples) or a built-in swimmer; returns
    {samples per SM: threads per sample} for the measured buckets."""
    out = (ctypes.c_int * 17)()
    if theta is not None:
        _dev(theta, torch.float64)
        check(lib().swimmer_autotune(h.ptr, int(steps), _ptr(theta), int(theta.shape[0]), out))
    else:
        check(lib().swimmer_autotune(h.ptr, int(steps), None, 0, out))
    return {k + 1: out[k] for k in range(17) if out[k] > 0}


def swimmer_tuning(h: Handle, precision=None, threads=None):
    """Get (threads=None) or set the launch-shape table of one precision: a list of 17
    threads-per-sample entries, entry k for batches of k + 1 samples per SM, 0 = heuristic;
    FP32C entries may carry SHAPE_WIDE or SHAPE_QUAD (two or four target blocks per pair
    unit)."""
    prec = h.cfg.precision if precision is None else precision
    buf = (ctypes.c_int * 17)()
    if threads is None:
        check(lib().swimmer_tuning(h.ptr, int(prec), buf, 0))
        return list(buf)
    vals = list(threads)
    if len(vals) != 17:
        raise ValueError("threads needs 17 entries")
    for k, v in enumerate(vals):
        buf[k] = int(v)
    check(lib().swimmer_tuning(h.ptr, int(prec), buf, 1))
    return vals


def swimmer_kernel_eval_noalloc(alpha, delta, r_max, r: torch.Tensor, precision=FP64, g1=None, g2=None,
                                stream=None):
    """Like swimmer_kernel_eval, without a handle: the library allocates nothing (its scratch
    is static device memory shared by all calls on the device).  Pass preallocated g1/g2
    to keep the whole call allocation-free on the Python side too."""
    _dev(r, torch.float64)
    g1 = torch.empty_like(r) if g1 is None else g1
    g2 = torch.empty_like(r) if g2 is None else g2
    # the kernel writes r.numel() doubles into each output on r's device
    for name, t in (("g1", g1), ("g2", g2)):
        _dev(t, torch.float64)
        if t.numel() != r.numel() or t.device != r.device:
            raise ValueError(f"{name} must hold {r.numel()} doubles on {r.device}")
    with torch.cuda.device(r.device):
        check(lib().swimmer_kernel_eval_noalloc(float(alpha), float(delta), float(r_max), r.numel(), _ptr(r),
                                                _ptr(g1), _ptr(g2), int(precision), _stream(stream)))
    return g1, g2


class ForwardGraph:
    """``forward_batch`` (or ``loglik_batch`` when ``obs`` is given) captured once in a CUDA
    graph and replayed: the table build, the work-queue reset and the persistent forward
    launch become one graph launch.  Write new parameters into ``self.theta`` (and sizes
    into ``self.n_pts``) in place, then ``replay()``; results land in the tensors of
    ``self.out``.  Capture happens after one eager call, so one-time set-up never runs
    inside the capture."""

    def __init__(self, h: Handle, theta, n_pts=None, want_traj=False, obs=None, sigma=None):
        self.h = h
        self.theta = theta.clone()
        self.n_pts = n_pts.clone() if n_pts is not None else None
        B = theta.shape[0]
        dev = theta.device
        if obs is None:
            traj = torch.empty((B, h.cfg.n_obs, 2), dtype=torch.float64, device=dev) if want_traj else None
            self.out = (traj, torch.empty(B, dtype=torch.float64, device=dev),
                        torch.empty(B, dtype=torch.int32, device=dev))
            call = lambda: forward_batch(h, self.theta, self.n_pts, want_traj, out=self.out)
        else:
            self.obs = obs
            self.out = (torch.empty(B, dtype=torch.float64, device=dev), torch.empty(B, dtype=torch.int32, device=dev))
            call = lambda: loglik_batch(h, self.theta, obs, sigma, n_pts=self.n_pts, out=self.out)
        call()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            call()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()
        return self.out
