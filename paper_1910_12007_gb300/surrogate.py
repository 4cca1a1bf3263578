"""Learned surrogate for delayed-acceptance TMCMC (not in the paper).

An MLP 5 -> 256 -> 256 -> 256 -> 80 (GELU, BF16 weights, FP32 accumulation) maps the
normalized inputs (alpha, log10 K_C, a, log10 K_T, omega) to 40 head positions (x, y), taken
every ``obs_stride``-th observation of the forward model.  The training set is generated by
the method itself (``forward_batch`` on prior draws); training runs the library's MLP
forward/backward/Adam kernels.  ``attach`` hands the trained network to a handle, after which
``tmcmc_stage(..., use_surrogate=True)`` screens proposals with it (delayed acceptance: the
plain forward model still decides every accepted move).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import api

N_OUT_TIMES = api.MLP_OUT // 2


@dataclass
class Surrogate:
    params: torch.Tensor      # FP32 master weights on the device
    in_lo: np.ndarray         # 5 input lower bounds (mapped to -1)
    in_hi: np.ndarray         # 5 input upper bounds (mapped to +1)
    out_mean: np.ndarray      # 80 output means
    out_std: np.ndarray       # 80 output standard deviations
    obs_stride: int
    log10_kt: float
    omega: float
    losses: list

    def attach(self, h: api.Handle):
        api.swimmer_surrogate_set(h, self.params, self.in_lo, self.in_hi, self.out_mean, self.out_std,
                                  self.obs_stride, self.log10_kt, self.omega)

    def predict(self, theta: torch.Tensor) -> torch.Tensor:
        """Head positions [B, 40, 2] predicted for theta [B, 3] (device FP64)."""
        x = self.inputs(theta)
        y = api.mlp_forward(self.params, x).double().cpu().numpy()
        y = self.out_mean + self.out_std * y
        return torch.tensor(y.reshape(-1, N_OUT_TIMES, 2))

    def inputs(self, theta: torch.Tensor) -> torch.Tensor:
        th = theta.double().cpu().numpy()
        v = np.concatenate([th, np.full((th.shape[0], 1), self.log10_kt), np.full((th.shape[0], 1), self.omega)], 1)
        span = np.where(self.in_hi > self.in_lo, self.in_hi - self.in_lo, 1.0)
        x = np.where(self.in_hi > self.in_lo, 2.0 * (v - self.in_lo) / span - 1.0, 0.0)
        return torch.tensor(x, dtype=torch.float32, device=theta.device)


def obs_stride_for(cfg: api.SwimmerConfig) -> int:
    n_obs = cfg.n_obs
    if n_obs < N_OUT_TIMES:
        raise ValueError(f"the surrogate needs at least {N_OUT_TIMES} observations, got {n_obs}")
    return n_obs // N_OUT_TIMES


def generate_training_set(h: api.Handle, thetas: torch.Tensor):
    """Forward runs of every row of thetas [n, 3] (device) in batches of b_max; returns the
    head trajectories [n, n_obs, 2] (device) and the status codes."""
    n = thetas.shape[0]
    B = h.cfg.b_max
    traj = torch.empty((n, h.cfg.n_obs, 2), dtype=torch.float64, device=thetas.device)
    status = torch.empty(n, dtype=torch.int32, device=thetas.device)
    for i in range(0, n, B):
        j = min(n, i + B)
        t, _, s = api.forward_batch(h, thetas[i:j].contiguous())
        traj[i:j] = t
        status[i:j] = s
    return traj, status


def init_params(seed, device):
    """He-style uniform initialization, biases zero (layout W1,b1,...,W4,b4, W[out][in])."""
    rng = np.random.default_rng(seed)
    layers = (api.MLP_IN, api.MLP_HIDDEN, api.MLP_HIDDEN, api.MLP_HIDDEN, api.MLP_OUT)
    parts = []
    for fi, fo in zip(layers[:-1], layers[1:]):
        lim = math.sqrt(3.0 / fi)
        parts.append(rng.uniform(-lim, lim, size=fo * fi))
        parts.append(np.zeros(fo))
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == api.MLP_NPARAM
    return torch.tensor(flat, device=device)


def train(h: api.Handle, thetas: torch.Tensor, prior_lo, prior_hi, epochs=60, batch=1024, lr=2e-3, seed=0,
          traj=None, status=None, log=None) -> Surrogate:
    """Generate (or take) forward runs at thetas, then fit the MLP with Adam (cosine-decayed
    learning rate).  Diverged runs are left out of the training set."""
    cfg = h.cfg
    dev = thetas.device
    stride = obs_stride_for(cfg)
    if traj is None:
        traj, status = generate_training_set(h, thetas)
    ok = status == 0
    rows = torch.arange(N_OUT_TIMES, device=dev) * stride + (stride - 1)
    Y = traj[ok][:, rows, :].reshape(-1, api.MLP_OUT)
    th = thetas[ok]
    log10_kt = math.log10(cfg.k_t) if cfg.k_t > 0 else 0.0
    in_lo = np.array([prior_lo[0], prior_lo[1], prior_lo[2], log10_kt, cfg.omega], dtype=np.float64)
    in_hi = np.array([prior_hi[0], prior_hi[1], prior_hi[2], log10_kt, cfg.omega], dtype=np.float64)
    Yc = Y.cpu().numpy()
    out_mean = Yc.mean(0)
    out_std = np.maximum(Yc.std(0), 1e-12)
    sur = Surrogate(init_params(seed, dev), in_lo, in_hi, out_mean, out_std, stride, log10_kt, cfg.omega, [])
    X = sur.inputs(th)
    T = torch.tensor((Yc - out_mean) / out_std, dtype=torch.float32, device=dev)
    n = X.shape[0]
    batch = min(batch, n)
    ws = api.mlp_workspace(batch, dev)
    m = torch.zeros_like(sur.params)
    v = torch.zeros_like(sur.params)
    grad = torch.empty_like(sur.params)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        ep_loss = 0.0
        for k in range(steps_per_epoch):
            idx = perm[k * batch:(k + 1) * batch]
            xb = X[idx].contiguous()
            tb = T[idx].contiguous()
            api.mlp_backward(sur.params, xb, tb, workspace=ws, grad=grad, loss=loss)
            step += 1
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))
            api.mlp_adam(sur.params, grad, m, v, step, lr_t)
            ep_loss += loss.item() if k == steps_per_epoch - 1 else 0.0
        sur.losses.append(ep_loss)
        if log is not None:
            log(ep, ep_loss)
    return sur


def validation_error(sur: Surrogate, traj: torch.Tensor, thetas: torch.Tensor, status: torch.Tensor):
    """Relative RMS error of the predicted head positions over held-out forward runs."""
    ok = status == 0
    rows = torch.arange(N_OUT_TIMES, device=traj.device) * sur.obs_stride + (sur.obs_stride - 1)
    ref = traj[ok][:, rows, :].cpu().numpy()
    pred = sur.predict(thetas[ok]).numpy()
    return float(np.sqrt(np.mean((pred - ref) ** 2)) / np.sqrt(np.mean((ref - ref.mean(0)) ** 2)))
