"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle.

This module holds none of the method's arithmetic: only a counter-based random
number generator (SplitMix64, Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) and the draws the method consumes as inputs (prior samples,
resampling and acceptance uniforms, proposal normals, observation noise).  Every random
number the method uses is generated here, on the host, and passed to both sides.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers
PRIOR, RESAMPLE, ACCEPT, ACCEPT2, PROPOSAL, NOISE, TRAIN = range(7)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, stream, stage):
    with np.errstate(over="ignore"):
        k = _mix(np.uint64(seed) * _GOLDEN + np.uint64(stream + 1))
        return _mix(k + np.uint64(stage + 1) * _GOLDEN)


def uniforms(seed, stream, stage, n):
    """n doubles in [0, 1) with 53 random bits: counter i -> mix(key + (i+1) * golden)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN
        z = _mix(_key(seed, stream, stage) + ctr)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed, stream, stage, n):
    """n standard normal doubles by the Box-Muller transform of 2n uniforms."""
    u = uniforms(seed, stream, stage, 2 * n)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def prior_samples(seed, lo, hi, n):
    """n draws from the box-uniform prior U[lo, hi] (one row per sample)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = uniforms(seed, PRIOR, 0, n * lo.size).reshape(n, lo.size)
    return lo + (hi - lo) * u


def stage_randoms(seed, stage, n, p):
    """The random inputs of one TMCMC stage: resampling uniforms [n], acceptance uniforms
    [2, n] (the second row is used by the second step of delayed acceptance) and proposal
    normals [n, p]."""
    u_res = uniforms(seed, RESAMPLE, stage, n)
    u_acc = np.stack([uniforms(seed, ACCEPT, stage, n), uniforms(seed, ACCEPT2, stage, n)])
    z = normals(seed, PROPOSAL, stage, n * p).reshape(n, p)
    return u_res, u_acc, z


def choice_n(seed, choices, n):
    """n values drawn uniformly from ``choices`` (uneven-size batches)."""
    c = np.asarray(choices)
    u = uniforms(seed, PRIOR, 7, n)
    return c[np.minimum((u * len(c)).astype(np.int64), len(c) - 1)]
