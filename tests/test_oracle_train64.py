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


def _kink_free(params, x, a1, h1, a2, layer, which, i, h):
    """True if moving parameter i of (layer, which) by +-h leaves the sign of
    every pre-activation it reaches unchanged."""
    w2 = np.asarray(params[1][0], np.float64)
    if layer == 2:
        return True
    fan_in = x.shape[1] if layer == 0 else h1.shape[1]
    unit = i // fan_in if which == 0 else i
    src = (x if layer == 0 else h1)[:, i % fan_in] if which == 0 else np.ones(x.shape[0])
    d = np.abs(h * src)                         # change of the unit's pre-activation per context
    pre = a1 if layer == 0 else a2
    if np.any(np.abs(pre[:, unit]) <= d):
        return False
    if layer == 1:
        return True
    d2 = d[:, None] * np.abs(w2[:, unit])[None, :] * (a1[:, unit] > 0)[:, None]
    return not np.any(np.abs(a2) <= d2)


@pytest.mark.slow
def test_gradient_vs_central_differences_cfg3_widths():
    # The training workload's own network (12-256-256-256) on its 2048-context
    # subset: cfg-3-style images, contexts sampled as the trainer's data.
    from paper_2207_05152_gb300 import train as T
    imgs = [synth.config_image(3, i) for i in range(2)]
    ctx, tgt = T.sample_contexts(imgs, 2048, 11)
    params = _params([12, 256, 256, 256], 12)
    grads, _ = train64.gradient(params, ctx, tgt)
    _, (x, a1, h1, a2, h2, z, lse) = train64.forward(params, ctx, tgt)
    checked = 0
    for layer in range(3):
        for which in range(2):
            g = grads[layer][which].reshape(-1)
            # the largest entries (where a dropped term or a wrong index
            # shows most) and a few seeded ones
            picks = list(np.argsort(-np.abs(g))[:2]) + list(synth.Rng(40 + 2 * layer + which).integers(2, 0, g.size - 1))
            for i in picks:
                i = int(i)
                theta = params[layer][which].reshape(-1)[i]
                h = 1e-6 * max(1.0, abs(theta))
                # with 2048 contexts and 256 units, a perturbation of h can
                # move some downstream pre-activation across zero; central
                # differences are only checked where none crosses (margin 2x)
                if not _kink_free(params, x, a1, h1, a2, layer, which, i, 2.0 * h):
                    continue
                fd = train64.finite_difference(params, ctx, tgt, layer, which, i, h)
                assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (layer, which, i, fd, g[i])
                checked += 1
    assert checked >= 16


def test_weighted_loss_pins():
    # the frequency-weighted loss (Sec. IV "Color Frequencies"): unit weights
    # give the plain loss; an integer weight k on a value is k copies of
    # every context with that target; central differences agree
    ctx, tgt = _batch(300, 31)
    params = _params([12, 24, 24, 256], 32, gain=2.0)
    ones = np.ones(256)
    l0, _ = train64.forward(params, ctx, tgt)
    l1, _ = train64.forward(params, ctx, tgt, ones)
    assert abs(l0 - l1) <= 1e-13 * l0
    g0, _ = train64.gradient(params, ctx, tgt)
    g1, _ = train64.gradient(params, ctx, tgt, ones)
    for a, b in zip(g0, g1):
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=1e-12, atol=1e-15)
    w = np.ones(256)
    w[np.unique(tgt)[::3]] = 3.0               # every third present value counts three times
    rep = np.concatenate([np.arange(tgt.size)] + [np.nonzero(w[tgt] == 3.0)[0]] * 2)
    lw, _ = train64.forward(params, ctx, tgt, w)
    lr, _ = train64.forward(params, ctx[rep], tgt[rep])
    assert abs(lw - lr) <= 1e-12 * lr
    gw, _ = train64.gradient(params, ctx, tgt, w)
    gr, _ = train64.gradient(params, ctx[rep], tgt[rep])
    for a, b in zip(gw, gr):
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=1e-9, atol=1e-14)
    _, (x, a1, h1, a2, h2, z, lse) = train64.forward(params, ctx, tgt, w)
    for layer, which in [(0, 1), (1, 0), (2, 0), (2, 1)]:
        g = gw[layer][which].reshape(-1)
        for i in np.argsort(-np.abs(g))[:2]:
            i = int(i)
            theta = params[layer][which].reshape(-1)[i]
            h = 1e-6 * max(1.0, abs(theta))
            if not _kink_free(params, x, a1, h1, a2, layer, which, i, 2.0 * h):
                continue
            fd = train64.finite_difference(params, ctx, tgt, layer, which, i, h, w)
            assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9


# --- 12-bit samples (Sec. IV "Higher Bit Depth": 4096 output neurons) -----

def _batch12(n, seed):
    from paper_2207_05152_gb300 import train as T
    imgs = [synth.phantom_image12(48, 40, seed + i) for i in range(2)]
    return T.sample_contexts(imgs, n, seed)


def test_twelve_bit_flat_network_costs_twelve_bits():
    ctx, tgt = _batch12(96, 51)
    assert ctx.dtype == np.uint16 and tgt.max() > 255
    params = _params([12, 16, 16, 4096], 52)
    params[2] = (np.zeros((4096, 16)), np.zeros(4096))
    loss, _ = train64.forward(params, ctx, tgt, bits=12)
    assert abs(loss - 12.0) < 1e-12
    grads, _ = train64.gradient(params, ctx, tgt, bits=12)
    counts = np.bincount(tgt, minlength=4096)
    want = (1.0 / 4096.0 - counts / len(tgt)) / np.log(2.0)
    assert np.allclose(grads[2][1], want, atol=1e-15)
    # a zero output layer passes no gradient to the hidden layers
    assert not np.any(grads[0][0]) and not np.any(grads[1][0]) and np.any(grads[2][0])


def test_twelve_bit_inputs_are_v_over_2048_minus_1():
    # a 12-bit context of multiples of 16 (16 u) is the 8-bit context u on
    # the input side: 16 u / 2048 - 1 = u / 128 - 1 exactly
    rng = synth.Rng(53)
    ctx8 = rng.integers(64 * 12, 0, 255).reshape(64, 12).astype(np.uint8)
    tgt = rng.integers(64, 0, 4095)
    ctx12 = ctx8.astype(np.uint16) * 16
    params = _params([12, 16, 16, 4096], 54, gain=2.0)
    l8, c8 = train64.forward(params, ctx8, tgt, bits=8)
    l12, c12 = train64.forward(params, ctx12, tgt, bits=12)
    assert l8 == l12 and np.array_equal(c8[0], c12[0])
    g8, _ = train64.gradient(params, ctx8, tgt, bits=8)
    g12, _ = train64.gradient(params, ctx12, tgt, bits=12)
    for a, b in zip(g8, g12):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    # the 8-bit scale on 12-bit samples is a different network input
    l_wrong, _ = train64.forward(params, ctx12, tgt, bits=8)
    assert abs(l_wrong - l12) > 1e-3


def test_twelve_bit_logits_match_the_coder():
    # the trained network is the one the 12-bit coder evaluates: the FP64
    # logits equal the oracle coder's FP32 logits of the same weights
    import oracle
    from paper_2207_05152_gb300 import model as M
    ctx, tgt = _batch12(200, 55)
    layers = synth.xavier_mlp([12, 32, 32, 4096], 56)
    _, cache = train64.forward(layers, ctx, tgt, bits=12)
    z64 = cache[5]
    z32 = oracle.logits(M.fp32_blob12(layers), ctx).astype(np.float64)
    assert np.max(np.abs(z64 - z32)) <= 2e-5 * max(1.0, np.max(np.abs(z64)))


@pytest.mark.parametrize("layer,which", [(0, 0), (1, 1), (2, 0), (2, 1)])
def test_twelve_bit_gradient_vs_central_differences(layer, which):
    ctx, tgt = _batch12(128, 57)
    params = _params([12, 16, 16, 4096], 58, gain=2.0)
    grads, _ = train64.gradient(params, ctx, tgt, bits=12)
    _, (x, a1, h1, a2, h2, z, lse) = train64.forward(params, ctx, tgt, bits=12)
    g = grads[layer][which].reshape(-1)
    picks = list(np.argsort(-np.abs(g))[:3]) + list(synth.Rng(60 + layer).integers(3, 0, g.size - 1))
    checked = 0
    for i in picks:
        i = int(i)
        theta = params[layer][which].reshape(-1)[i]
        h = 1e-6 * max(1.0, abs(theta))
        if not _kink_free(params, x, a1, h1, a2, layer, which, i, 2.0 * h):
            continue
        fd = train64.finite_difference(params, ctx, tgt, layer, which, i, h, bits=12)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])
        checked += 1
    assert checked >= 3
