"""The allocation-free kernel-function entry point (swimmer_kernel_eval_noalloc) against the
handle-based swimmer_kernel_eval.

It serves callers that may not allocate device memory (fixed start-up memory budgets): its
scratch is static device memory shared by all calls on a device.  This file is collected last so that a run stopping at the first failure
has already run every other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1910_12007_gb300 as g  # noqa: E402

DEV = torch.device("cuda:0")


def _points(delta, r_max, seed):
    rng = np.random.default_rng(seed)
    r = np.concatenate([[0.0, 0.3 * delta, delta, 0.9 * r_max], rng.uniform(0, r_max, 40), rng.uniform(0, 4 * delta, 20)])
    return torch.tensor(r, dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-6)])
def test_noalloc_matches_handle_path_on_consecutive_calls(precision, tol):
    delta, r_max = 1.5 / 127, 1.25
    h = g.swimmer_init(g.SwimmerConfig(n_max=128, b_max=1, steps=1, obs_every=1))
    # two different samples in a row: the second call must not see the first one's tables
    for alpha, seed in [(2.5, 1), (0.4, 2)]:
        r = _points(delta, r_max, seed)
        ref1, ref2 = g.swimmer_kernel_eval(h, alpha, delta, r_max, r, precision)
        out1 = torch.full_like(r, float("nan"))
        out2 = torch.full_like(r, float("nan"))
        g.swimmer_kernel_eval_noalloc(alpha, delta, r_max, r, precision, g1=out1, g2=out2)
        torch.cuda.synchronize()
        a1, a2, b1, b2 = (t.cpu().numpy() for t in (out1, out2, ref1, ref2))
        assert np.all(np.isfinite(a1)) and np.all(np.isfinite(a2))
        s1 = np.maximum(np.abs(b1), 0.05)
        assert np.max(np.abs(a1 - b1) / s1) < tol
        assert np.max(np.abs(a2 - b2) / np.abs(b2)) < tol
    h.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    r = torch.zeros(4, dtype=torch.float64, device=DEV)
    with pytest.raises(RuntimeError, match="beyond"):
        g.swimmer_kernel_eval_noalloc(1.0, 1e-4, 1.0, r)  # r_max/delta = 1e4 > 4000


def test_noalloc_leaves_device_memory_unchanged():
    """After the first call on the device (its one-time set-up), further calls with
    preallocated outputs take no device memory: the free memory the driver reports stays the
    same over repeated calls."""
    delta, r_max = 1.5 / 127, 1.25
    r = _points(delta, r_max, 3)
    out1, out2 = torch.empty_like(r), torch.empty_like(r)
    g.swimmer_kernel_eval_noalloc(1.0, delta, r_max, r, 1, g1=out1, g2=out2)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for alpha in (0.5, 3.0, 7.5, 0.0):
        for precision in (0, 1):
            g.swimmer_kernel_eval_noalloc(alpha, delta, r_max, r, precision, g1=out1, g2=out2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.isfinite(out1).all() and torch.isfinite(out2).all()


def test_noalloc_rejects_bad_outputs_before_launch():
    r = torch.linspace(0.0, 1.0, 16, dtype=torch.float64, device=DEV)
    good = torch.full_like(r, float("nan"))
    bad = [torch.empty(16, dtype=torch.float32, device=DEV),  # wrong dtype
           torch.empty(15, dtype=torch.float64, device=DEV),  # too short
           torch.empty(32, dtype=torch.float64, device=DEV)[::2],  # not contiguous
           torch.empty(16, dtype=torch.float64)]  # host memory
    for b in bad:
        with pytest.raises((TypeError, ValueError)):
            g.swimmer_kernel_eval_noalloc(1.0, 0.02, 1.0, r, 0, g1=good, g2=b)
    torch.cuda.synchronize()
    assert torch.isnan(good).all()  # nothing ran
