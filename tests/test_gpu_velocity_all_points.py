"""Per-step FP32 velocities at EVERY point against the oracle (Eq. BrV), through the C ABI.

Two forward runs of the same batch, K and K + 1 Euler steps, return their final states
(positions and forces).  The FP32 kernel's velocity at step K is its displacement over the
last step divided by dt; the oracle evaluates Eq. BrV with the exact forces of Eq. Fenergy at
the same positions (the GPU run's own state after K steps).  At N = 128 and N = 256 the runs
are long enough for the filament to bend (2e4 steps), so separations point in every
direction; at N = 1024 the state is the large sweep's own nearly straight regime (its whole
run spans 1.2e-4 time units).  The
tolerance is the FP32 kernel's 1e-4 relative on velocities, against the largest velocity of
the sample, for every launch shape the autotuner chooses from.  The kernel's forces (Eq.
Fenergy, an intermediate) are checked at 1e-3 of the largest force plus 1e-3 absolute: the
bending force is a second difference of stencil terms of size 2 K_C (zeta - zeta^)/ds, and FP32
rounding of zeta and zeta^ (values up to a eta^2) leaves an absolute floor of a few 1e-4 at
N = 128 that dominates once the filament has relaxed and its net forces are small.  One check evaluates two
target rows directly from the radial-integral definition of the kernel functions instead of
the oracle's interpolation table.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic
from oracle import brinkmanlet as bk
from oracle import swimmer as sw

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1910_12007_gb300 as g  # noqa: E402

DEV = torch.device("cuda:0")


def _states(p, th, steps, shape, b_max):
    """Final states of the batch th after `steps` and `steps + 1` Euler steps."""
    out = []
    for k in (steps, steps + 1):
        cfg = g.SwimmerConfig(n_max=p.n, b_max=b_max, length=p.length, dt=p.dt, k_t=p.k_t, steps=k, obs_every=k,
                              precision=g.FP32C)
        h = g.swimmer_init(cfg)
        g.swimmer_tuning(h, g.FP32C, [shape] * 17)
        _, _, status, state = g.forward_batch_state(h, torch.tensor(th, device=DEV))
        torch.cuda.synchronize()
        assert np.all(status.cpu().numpy() == 0)
        out.append(state.cpu().numpy())
        h.close()
    return out


def _check(p, theta, s0, s1, steps):
    q = p.with_theta(tuple(theta))
    X = s0[:, :2]
    v_gpu = (s1[:, :2] - X) / q.dt
    F = sw.forces(X, q, steps * q.dt)
    v = sw.velocity(X, F, sw.kernel_table(q), q.mu)
    err_v = np.max(np.abs(v_gpu - v)) / np.max(np.abs(v))
    err_f = np.max(np.abs(s0[:, 2:] - F)) / (np.max(np.abs(F)) + 1.0)
    return err_v, err_f, v_gpu, F


# the TMCMC workload's swimmer: N = 128, dt = 1e-4/64, 1024 samples in one launch
N128 = sw.SwimmerParams(n=128, dt=1e-4 / 64, k_t=1e3)


@pytest.fixture(scope="module")
def batch128():
    th = synthetic.prior_samples(31, (0.0, -1.0, 0.05), (10.0, 0.2, 0.2), 1024)
    th[0] = (1.0, 0.0, 0.1)
    return th


@pytest.mark.parametrize("shape", [128, 256, 512, 128 | g.SHAPE_WIDE, 256 | g.SHAPE_WIDE])
def test_all_point_velocities_n128(shape, batch128):
    steps = 20000
    s0, s1 = _states(N128, batch128, steps, shape, 1024)
    for b in (0, 1, 511, 1023):
        err_v, err_f, v_gpu, F = _check(N128, batch128[b], s0[b], s1[b], steps)
        assert err_v < 1e-4, (shape, b, err_v)
        assert err_f < 1e-3, (shape, b, err_f)
    if shape == 128:
        # two target rows from the pointwise definition of g1, g2 (no table on either side)
        q = N128.with_theta(tuple(batch128[0]))
        X = s0[0][:, :2]
        F = sw.forces(X, q, steps * q.dt)
        pointwise = np.vectorize(lambda r: bk.kernel_g(r, q.alpha, q.delta))
        rows = [0, q.n - 1]
        v_pt, _ = sw.flow_field(X, F, X[rows], lambda r: pointwise(r), q.delta, q.mu)
        v_gpu = (s1[0][rows, :2] - X[rows]) / q.dt
        assert np.max(np.abs(v_gpu - v_pt)) < 1e-4 * np.max(np.abs(v_pt))


# a swimmer of 8 blocks of 32 points (the smallest with four-target units): N = 256 at the
# uneven batch's ds = 1/255 and dt = 1e-4/512
N256 = sw.SwimmerParams(n=256, dt=1e-4 / 512, k_t=1e3)


@pytest.mark.parametrize("shape", [256 | g.SHAPE_QUAD, 512 | g.SHAPE_QUAD, 256 | g.SHAPE_WIDE])
def test_all_point_velocities_n256(shape):
    th = synthetic.prior_samples(32, (0.0, -1.0, 0.05), (10.0, 0.0, 0.2), 256)
    steps = 20000
    s0, s1 = _states(N256, th, steps, shape, 256)
    for b in (0, 128, 255):
        err_v, err_f, _, _ = _check(N256, th[b], s0[b], s1[b], steps)
        assert err_v < 1e-4, (shape, b, err_v)
        assert err_f < 1e-3, (shape, b, err_f)


# the large sweep's swimmer: N = 1024, dt = 1e-4/2^15, 256 samples, alpha in [0, 50]
N1024 = sw.SwimmerParams(n=1024, dt=1e-4 / 2 ** 15, k_t=1e3)


@pytest.fixture(scope="module")
def batch1024():
    return synthetic.prior_samples(3000, (0.0, -1.0, 0.05), (50.0, 0.0, 0.2), 256)


@pytest.mark.parametrize("shape", [512 | g.SHAPE_QUAD, 512 | g.SHAPE_WIDE, 512, 256 | g.SHAPE_QUAD, 128])
def test_all_point_velocities_n1024(shape, batch1024):
    steps = 2000
    s0, s1 = _states(N1024, batch1024, steps, shape, 256)
    for b in (0, 255):
        err_v, err_f, _, _ = _check(N1024, batch1024[b], s0[b], s1[b], steps)
        assert err_v < 1e-4, (shape, b, err_v)
        assert err_f < 1e-3, (shape, b, err_f)
