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
