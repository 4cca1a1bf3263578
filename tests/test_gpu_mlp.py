"""GPU parity of the surrogate MLP kernels (forward, backward, Adam) against the FP64
oracle MLP evaluated with the same BF16-rounded weights and, in the 256-wide layers, the
same BF16 operands (the tensor-core products round activations and output gradients to
BF16 as they enter; the oracle rounds the same factors and sums exactly).  Tolerances: the
GPU sums in FP32, and where an FP32 activation lies within rounding of a BF16 boundary the
two sides may round it to neighbouring BF16 values (2^-8 apart), which moves a product by
about 4e-3 of one term."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as om

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1910_12007_gb300 as g  # noqa: E402

DEV = torch.device("cuda:0")


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def _unflat(v):
    out, o = [], 0
    for fi, fo in zip(om.LAYERS[:-1], om.LAYERS[1:]):
        W = v[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = v[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def _setup(n, seed=0):
    rng = np.random.default_rng(seed)
    params = om.init_params(rng)
    params = [(W, rng.normal(0, 0.1, size=b.shape)) for W, b in params]
    flat = _flat(params).astype(np.float32)
    rounded = [(om.bf16_round(W.astype(np.float32)), b.astype(np.float32).astype(np.float64))
               for W, b in _unflat(flat.astype(np.float64))]
    x = rng.uniform(-1, 1, size=(n, 5)).astype(np.float32)
    t = rng.normal(size=(n, 80)).astype(np.float32)
    return flat, rounded, x, t


@pytest.mark.parametrize("n", [1, 37, 256, 1000])
def test_mlp_forward_matches_oracle(n):
    flat, rounded, x, t = _setup(n)
    y = g.mlp_forward(torch.tensor(flat, device=DEV), torch.tensor(x, device=DEV)).cpu().numpy()
    ref = om.forward(rounded, x.astype(np.float64), bf16_operands=True)
    assert np.max(np.abs(y - ref)) < 2e-3 * np.max(np.abs(ref))
    # and the BF16 operands are what the GPU computes: the unrounded network is farther away
    full = om.forward(rounded, x.astype(np.float64))
    assert np.max(np.abs(y - ref)) < 0.5 * np.max(np.abs(y - full))


@pytest.mark.parametrize("n", [5, 300])
def test_mlp_backward_matches_oracle(n):
    flat, rounded, x, t = _setup(n, 3)
    grad, loss = g.mlp_backward(torch.tensor(flat, device=DEV), torch.tensor(x, device=DEV),
                                torch.tensor(t, device=DEV))
    grad = grad.cpu().numpy().astype(np.float64)
    ref = om.backward(rounded, x.astype(np.float64), t.astype(np.float64), bf16_operands=True)
    ref_flat = _flat(ref)
    y_ref = om.forward(rounded, x.astype(np.float64), bf16_operands=True)
    assert abs(loss.item() - float(np.mean((y_ref - t) ** 2))) < 1e-4 * float(np.mean((y_ref - t) ** 2))
    # per layer, against that layer's largest gradient entry
    o = 0
    for W, b in ref:
        for part in (W.ravel(), b):
            seg = grad[o:o + part.size]
            o += part.size
            assert np.max(np.abs(seg - part)) < 2e-3 * np.max(np.abs(part)), (part.size,)


def test_mlp_backward_deterministic():
    flat, rounded, x, t = _setup(200, 4)
    args = [torch.tensor(a, device=DEV) for a in (flat, x, t)]
    g1, _ = g.mlp_backward(*args)
    g2, _ = g.mlp_backward(*args)
    assert torch.equal(g1, g2)


def test_adam_matches_oracle():
    flat, rounded, x, t = _setup(64, 5)
    rng = np.random.default_rng(1)
    grad = rng.normal(size=flat.size).astype(np.float32)
    p = torch.tensor(flat, device=DEV)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    gt = torch.tensor(grad, device=DEV)
    g.mlp_adam(p, gt, m, v, 1, 1e-3)
    g.mlp_adam(p, gt, m, v, 2, 1e-3)
    P = [(flat.astype(np.float64), np.zeros(1))]
    G = [(grad.astype(np.float64), np.zeros(1))]
    Z = [(np.zeros(flat.size), np.zeros(1))]
    P1, M1, V1 = om.adam_step(P, G, Z, Z, 1, lr=1e-3)
    P2, _, _ = om.adam_step(P1, G, M1, V1, 2, lr=1e-3)
    assert np.max(np.abs(p.cpu().numpy() - P2[0][0])) < 1e-6


def test_training_reduces_loss():
    n = 512
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, size=(n, 5)).astype(np.float32)
    t = np.concatenate([np.sin(2 * x[:, :1] + k * 0.1) for k in range(80)], axis=1).astype(np.float32)
    flat = _flat(om.init_params(rng)).astype(np.float32)
    p = torch.tensor(flat, device=DEV)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    X, T = torch.tensor(x, device=DEV), torch.tensor(t, device=DEV)
    ws = g.mlp_workspace(n, DEV)
    losses = []
    for step in range(1, 301):
        grad, loss = g.mlp_backward(p, X, T, workspace=ws)
        g.mlp_adam(p, grad, m, v, step, 2e-3)
        losses.append(loss.item())
    assert losses[-1] < 0.05 * losses[0]
