"""FP64 reference multilayer perceptron for the learned surrogate (oracle; tests only).

The surrogate is not in the paper; it is a fully connected network
5 -> 256 -> 256 -> 256 -> 80 with GELU activations on the hidden layers, mapping
normalized (alpha, log10 K_C, a, log10 K_T, omega) to 40 normalized head positions
(x, y).  Loss: mean squared error over all outputs of a batch.  Optimizer: Adam
(Kingma & Ba 2015) with bias correction.

Parameters are a list of (W[out, in], b[out]).  GELU(x) = x Phi(x) = x (1 + erf(x/sqrt 2))/2.

``bf16_operands=True`` gives the precision of a network whose 256-wide layers run as BF16
products with wide accumulation: for every layer after the first, both factors of each
product (activations or output gradients, and the weights, which the caller rounds) are
rounded to BF16 first, and the sums are exact here.  The first layer (5 inputs) keeps its
inputs unrounded.

Pins (in tests/test_oracle_tmcmc.py, the MLP tests): gradients against central finite differences of the
loss; GELU derivative against finite differences; an Adam step against its textbook
formula on one scalar.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

LAYERS = (5, 256, 256, 256, 80)


def init_params(rng, layers=LAYERS):
    """He-style uniform init: W ~ U(-sqrt(6/in), sqrt(6/in)) / sqrt(2), b = 0."""
    ps = []
    for fi, fo in zip(layers[:-1], layers[1:]):
        lim = math.sqrt(3.0 / fi)
        ps.append((rng.uniform(-lim, lim, size=(fo, fi)), np.zeros(fo)))
    return ps


def gelu(x):
    return 0.5 * x * (1.0 + special.erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + special.erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(params, x, keep=False, bf16_operands=False):
    """x[batch, 5] -> y[batch, 80]; with keep=True also the pre-activations."""
    h = np.asarray(x, dtype=np.float64)
    pre = []
    acts = [h]
    for li, (W, b) in enumerate(params):
        hin = bf16_round(h) if bf16_operands and li > 0 else h
        z = hin @ W.T + b
        pre.append(z)
        h = gelu(z) if li < len(params) - 1 else z
        acts.append(h)
    return (h, pre, acts) if keep else h


def loss(params, x, t):
    y = forward(params, x)
    return float(np.mean((y - t) ** 2))


def backward(params, x, t, bf16_operands=False):
    """Gradients of the mean squared error loss with respect to every W and b (with
    bf16_operands, those of the rounded products, differentiated as if the rounding were
    the identity)."""
    y, pre, acts = forward(params, x, keep=True, bf16_operands=bf16_operands)
    g = 2.0 * (y - t) / y.size
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li < len(params) - 1:
            g = g * gelu_grad(pre[li])
        r = bf16_operands and li > 0
        gr = bf16_round(g) if r else g
        grads[li] = (gr.T @ (bf16_round(acts[li]) if r else acts[li]), g.sum(axis=0))
        g = gr @ W
    return grads


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in place on copies); step counts from 1."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        layer = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = beta1 * mm + (1 - beta1) * g
            vv = beta2 * vv + (1 - beta2) * g * g
            mh = mm / (1 - beta1 ** step)
            vh = vv / (1 - beta2 ** step)
            layer.append((p - lr * mh / (np.sqrt(vh) + eps), mm, vv))
        out_p.append((layer[0][0], layer[1][0]))
        out_m.append((layer[0][1], layer[1][1]))
        out_v.append((layer[0][2], layer[1][2]))
    return out_p, out_m, out_v


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (round half to even), returned as FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def surrogate_inputs(theta, in_lo, in_hi, log10_kt, omega):
    """The network's inputs for theta rows (alpha, log10 K_C, a[, s]): the vector
    (alpha, log10 K_C, a, log10 K_T, omega) mapped affinely from [in_lo, in_hi] to [-1, 1]
    (0 where the range is empty), rounded to FP32 as the network receives them."""
    th = np.asarray(theta, dtype=np.float64)
    v = np.concatenate([th[:, :3], np.full((th.shape[0], 1), log10_kt), np.full((th.shape[0], 1), omega)], 1)
    lo = np.asarray(in_lo, dtype=np.float64)
    hi = np.asarray(in_hi, dtype=np.float64)
    span = hi - lo
    x = np.where(span > 0, 2.0 * (v - lo) / np.where(span > 0, span, 1.0) - 1.0, 0.0)
    return x.astype(np.float32).astype(np.float64)


def surrogate_loglik(params, theta, in_lo, in_hi, out_mean, out_std, obs_stride, log10_kt, omega, D, sigma):
    """Surrogate log-likelihood used by delayed acceptance (not in the paper).

    The network (its 256-wide layers as BF16 products, ``forward(..., bf16_operands=True)``)
    predicts the head position at 40 observation times, rows
    o * obs_stride + obs_stride - 1 of the observation record D [n_obs, 2]:
    p = out_mean + out_std * y.  The misfit over those rows is scaled to the full record,
    J = (n_obs / 40) sum |D_row - p|^2, and enters the Gaussian log-likelihood of Sec. 3.1
    (Eqs. likelihood, fitness): -(m/2) ln(2 pi sigma^2) - J / (2 sigma^2), m = 2 n_obs.
    With a fourth unknown the sample's sigma is theta[3] times sigma."""
    th = np.asarray(theta, dtype=np.float64)
    y = forward(params, surrogate_inputs(th, in_lo, in_hi, log10_kt, omega), bf16_operands=True)
    pred = np.asarray(out_mean)[None, :] + np.asarray(out_std)[None, :] * y
    D = np.asarray(D, dtype=np.float64)
    n_obs = D.shape[0]
    k = pred.shape[1] // 2
    rows = np.arange(k) * obs_stride + obs_stride - 1
    J = np.sum((D[rows][None, :, :] - pred.reshape(-1, k, 2)) ** 2, axis=(1, 2)) * (n_obs / k)
    s = sigma * th[:, 3] if th.shape[1] == 4 else np.full(th.shape[0], float(sigma))
    return -n_obs * np.log(2.0 * math.pi * s * s) - 0.5 * J / (s * s)
