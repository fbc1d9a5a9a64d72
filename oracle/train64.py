"""FP64 reference of the training objective (test infrastructure only).

The paper trains the density-estimation network with categorical
cross-entropy reported in bits per pixel (Sec. III-A, Table I: "vloss in
bpp").  Reading: for a batch of B (context, target) pairs the loss is
    L = (1/B) * sum_b -log2 softmax(z_b)[y_b],
with z = W3 relu(W2 relu(W1 x + b1) + b2) + b3 and x = v/128 - 1 for 8-bit
samples (256 outputs).  For 12-bit samples (Sec. IV "Higher Bit Depth": one
12-bit channel, 4096 output neurons) the same expression runs with
x = v/2048 - 1 and 4096 outputs; the output count is W3's row count.  The
gradient is the textbook adjoint of that expression: dL/dz = (softmax(z) -
onehot(y)) / (B ln 2), then the dense-layer and ReLU adjoints.  Adam (Kingma
and Ba 2015) with bias correction is the optimiser reading.  Everything here
is float64 numpy; matrix products use numpy's matmul as a library primitive.

The frequency-weighted loss (Sec. IV "Color Frequencies": the loss weighted
by value frequency, so that rare values count more) takes a weight w_v per
target value v: L = sum_b w_{y_b} * -log2 softmax(z_b)[y_b] / sum_b w_{y_b}.
Its gradient replaces 1/B by w_{y_b} / sum w.  With every w_v = 1 it is the
plain loss, and an integer weight k on a context is the same as k copies of
it in the batch.
"""
from __future__ import annotations

import numpy as np

LN2 = np.log(2.0)


def features(ctx, bits: int = 8) -> np.ndarray:
    """Network inputs v / 2^(bits-1) - 1: v/128 - 1 for 8-bit samples,
    v/2048 - 1 for 12-bit ones."""
    return np.asarray(ctx).astype(np.float64) / float(1 << (bits - 1)) - 1.0


def _row_weights(tgt, weights):
    """Per-context loss weights w_{y_b} / sum_b w_{y_b} (1/B unweighted)."""
    y = np.asarray(tgt, np.int64)
    if weights is None:
        return np.full(y.size, 1.0 / y.size)
    w = np.asarray(weights, np.float64)[y]
    return w / w.sum()


def forward(params, ctx_u8, tgt, weights=None, bits: int = 8):
    """params: [(W1, b1), (W2, b2), (W3, b3)] (any float dtype); weights:
    None, or one loss weight per target value; bits: the sample depth of the
    contexts (8 or 12).  Returns (loss_bits, cache)."""
    (w1, b1), (w2, b2), (w3, b3) = [(np.asarray(w, np.float64), np.asarray(b, np.float64))
                                    for w, b in params]
    x = features(ctx_u8, bits)
    a1 = x @ w1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3.T + b3
    zm = z.max(axis=1, keepdims=True)
    lse = zm[:, 0] + np.log(np.exp(z - zm).sum(axis=1))
    B = z.shape[0]
    nll = lse - z[np.arange(B), np.asarray(tgt, np.int64)]
    loss = nll.mean() / LN2 if weights is None else float((_row_weights(tgt, weights) * nll).sum()) / LN2
    return loss, (x, a1, h1, a2, h2, z, lse)


def gradient(params, ctx_u8, tgt, weights=None, bits: int = 8):
    """Analytic FP64 gradient: [(dW1, db1), (dW2, db2), (dW3, db3)], loss."""
    loss, (x, a1, h1, a2, h2, z, lse) = forward(params, ctx_u8, tgt, weights, bits)
    w1, w2, w3 = [np.asarray(p[0], np.float64) for p in params]
    B = z.shape[0]
    p = np.exp(z - lse[:, None])
    dz = p
    dz[np.arange(B), np.asarray(tgt, np.int64)] -= 1.0
    if weights is None:
        dz /= B * LN2
    else:
        dz *= (_row_weights(tgt, weights) / LN2)[:, None]
    dw3 = dz.T @ h2
    db3 = dz.sum(axis=0)
    dh2 = dz @ w3
    da2 = dh2 * (a2 > 0)
    dw2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    dh1 = da2 @ w2
    da1 = dh1 * (a1 > 0)
    dw1 = da1.T @ x
    db1 = da1.sum(axis=0)
    return [(dw1, db1), (dw2, db2), (dw3, db3)], loss


def finite_difference(params, ctx_u8, tgt, layer: int, which: int, index, h: float, weights=None, bits: int = 8):
    """Central difference (L(theta + h e) - L(theta - h e)) / 2h for one
    parameter (layer 0..2, which 0 = weight / 1 = bias, flat index)."""
    def loss_with(delta):
        ps = [[np.array(w, np.float64, copy=True), np.array(b, np.float64, copy=True)]
              for w, b in params]
        ps[layer][which].reshape(-1)[index] += delta
        return forward([tuple(q) for q in ps], ctx_u8, tgt, weights, bits)[0]
    return (loss_with(h) - loss_with(-h)) / (2.0 * h)


def adam_step(theta, grad, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in float64; step counts from 1.  Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
