"""Pins of the FP64 training reference (oracle/train64.py).

The loss is the categorical cross-entropy in bits (Sec. III-A, "vloss in
bpp"); its analytic gradient is checked against central finite differences,
and the closed forms of a flat network (8 bits, bias gradient from target
frequencies) and of Adam's first step are checked directly."""
import numpy as np
import pytest

import synth
from oracle import train64


def _batch(n, seed):
    rng = synth.Rng(seed)
    ctx = rng.integers(n * 12, 0, 255).reshape(n, 12).astype(np.uint8)
    tgt = rng.integers(n, 0, 255)
    return ctx, tgt


def _params(widths, seed, gain=1.0):
    layers = synth.xavier_mlp(widths, seed)
    rng = synth.Rng(seed + 1)
    out = []
    for w, b in layers:
        out.append((w.astype(np.float64) * gain, 0.1 * rng.normal(b.size)))
    return out


def test_flat_network_costs_eight_bits():
    ctx, tgt = _batch(64, 1)
    params = _params([12, 16, 16, 256], 2)
    params[2] = (np.zeros((256, 16)), np.zeros(256))
    loss, _ = train64.forward(params, ctx, tgt)
    assert abs(loss - 8.0) < 1e-12
    grads, _ = train64.gradient(params, ctx, tgt)
    counts = np.bincount(tgt, minlength=256)
    want = (1.0 / 256.0 - counts / len(tgt)) / np.log(2.0)
    assert np.allclose(grads[2][1], want, atol=1e-15)


@pytest.mark.parametrize("layer,which", [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)])
def test_gradient_vs_central_differences(layer, which):
    ctx, tgt = _batch(256, 3)
    params = _params([12, 32, 32, 256], 4, gain=2.0)
    grads, _ = train64.gradient(params, ctx, tgt)
    _, (x, a1, h1, a2, h2, z, lse) = train64.forward(params, ctx, tgt)
    g = grads[layer][which].reshape(-1)
    rng = synth.Rng(10 * layer + which)
    idx = rng.integers(12, 0, g.size - 1)
    for i in idx:
        theta = params[layer][which].reshape(-1)[i]
        h = 1e-6 * max(1.0, abs(theta))
        fd = train64.finite_difference(params, ctx, tgt, layer, which, int(i), h)
        # skip parameters feeding a unit whose pre-activation sits at a kink
        if layer < 2:
            pre = a1 if layer == 0 else a2
            unit = i // (12 if layer == 0 else 32) if which == 0 else i
            if np.min(np.abs(pre[:, unit])) < 1e-4:
                continue
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5, 0.0])
    grad = np.array([0.3, -1e-3, 0.0, 5.0])
    t, m, v = train64.adam_step(theta, grad, np.zeros(4), np.zeros(4), 1)
    # After one step the bias-corrected moments are g and g^2, so the update
    # is lr * g / (|g| + eps).
    want = theta - 1e-3 * grad / (np.abs(grad) + 1e-8)
    assert np.allclose(t, want, rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * grad) and np.allclose(v, 0.001 * grad * grad)
