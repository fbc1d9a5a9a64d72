"""12-bit training (Sec. IV "Higher Bit Depth": one 12-bit channel, 4096
output neurons) on the GPU against the FP64 reference (oracle/train64.py,
bits=12: inputs v/2048 - 1, the 4096-way cross-entropy in bits).

The output layer's products go to an FP32 buffer and a row-wise kernel takes
the softmax over 4096 values; everything else is the 8-bit trainer's.  The
same norm-wise bars as there: FP32 and split BF16 within 1e-3 of FP64 per
parameter tensor, plain BF16 reported at its own (bf16 operand) accuracy."""
import numpy as np
import pytest
import torch

import synth
from oracle import train64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300 import train
    return train


def _images(seed, n=3, size=(96, 80)):
    return [synth.phantom_image12(size[0], size[1], seed + i) for i in range(n)]


def _data(T, n, seed, widths=(12, 128, 128, 4096)):
    ctx, tgt = T.sample_contexts(_images(seed), n, seed)
    assert ctx.dtype == np.uint16 and tgt.max() > 255
    layers = synth.xavier_mlp(list(widths), seed)
    rng = synth.Rng(seed + 100)
    layers = [(w, (0.05 * rng.normal(b.size)).astype(np.float32)) for w, b in layers]
    return layers, ctx, tgt


def _dev(a):
    # u16 samples travel as int16 bits (torch's uint16 support varies)
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).cuda()


def _rel(g, ref):
    return float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30))


def _grads(T, mode, layers, ctx, tgt, max_batch=None, weights=None):
    tr = T.Trainer(layers, mode, max_batch=max_batch or len(tgt))
    if weights is not None:
        tr.set_value_weights(weights)
    loss, g = tr.backward(_dev(ctx), _dev(tgt))
    torch.cuda.synchronize()
    assert tr.status() == 0
    out = float(loss.item()), T.unflatten(g.cpu().numpy(), tr.h1, tr.h2, tr.n_in, tr.n_out)
    tr.close()
    return out


@pytest.mark.parametrize("mode,tol", [("fp32", 2e-4), ("bf16x3", 1e-3), ("bf16", 3e-2)])
def test_12bit_gradient_against_fp64(T, mode, tol):
    # 2048 contexts of 12-bit phantoms, the 12-bit coder's 12-128-128-4096
    layers, ctx, tgt = _data(T, 2048, 41)
    loss, g = _grads(T, mode, layers, ctx, tgt)
    ref, loss64 = train64.gradient(layers, ctx, tgt, bits=12)
    errs = [(_rel(gw, rw), _rel(gb, rb)) for (gw, gb), (rw, rb) in zip(g, ref)]
    print(mode, "loss", loss, "fp64", loss64, "norm-wise rel errors (W, b) per layer:", errs)
    assert abs(loss - loss64) <= 1e-3 * loss64
    for ew, eb in errs:
        assert ew < tol and eb < tol


@pytest.mark.parametrize("mode,tol", [("fp32", 2e-4), ("bf16x3", 1e-3)])
def test_12bit_ragged_weighted_and_chunked(T, mode, tol):
    # 1300 contexts (a ragged last tile) through a trainer sized for 512
    # (chunks of 512, 512, 276), with the frequency-weighted loss over the
    # 4096 values (Sec. IV "Color Frequencies")
    layers, ctx, tgt = _data(T, 1300, 43, widths=(12, 64, 48, 4096))
    w = T.frequency_weights(_images(43))
    assert w.size == 4096
    loss, g = _grads(T, mode, layers, ctx, tgt, max_batch=512, weights=w)
    ref, loss64 = train64.gradient(layers, ctx, tgt, w, bits=12)
    assert abs(loss - loss64) <= 1e-3 * loss64
    for (gw, gb), (rw, rb) in zip(g, ref):
        assert _rel(gw, rw) < tol and _rel(gb, rb) < tol


def test_12bit_flat_network_costs_twelve_bits(T):
    layers, ctx, tgt = _data(T, 700, 45, widths=(12, 32, 32, 4096))
    layers[2] = (np.zeros((4096, 32), np.float32), np.zeros(4096, np.float32))
    loss, g = _grads(T, "bf16x3", layers, ctx, tgt)
    assert abs(loss - 12.0) < 1e-5
    counts = np.bincount(tgt, minlength=4096)
    want = (1.0 / 4096.0 - counts / len(tgt)) / np.log(2.0)
    assert np.allclose(g[2][1], want, atol=1e-6)


def test_12bit_apply_of_own_gradient_is_the_step(T):
    layers, ctx, tgt = _data(T, 1000, 47, widths=(12, 64, 64, 4096))
    c, t = _dev(ctx), _dev(tgt)
    a = T.Trainer(layers, "bf16x3", max_batch=1000)
    b = T.Trainer(layers, "bf16x3", max_batch=1000)
    for _ in range(3):
        a.step(c, t)
        _, g = b.backward(c, t)
        b.apply(g)
    pa, pb = a.params(), b.params()
    torch.cuda.synchronize()
    assert torch.equal(pa, pb)
    assert a.status() == 0 and b.status() == 0
    a.close()
    b.close()


def test_12bit_sample_above_4095_is_flagged(T):
    from paper_2207_05152_gb300 import _lib
    layers, ctx, tgt = _data(T, 256, 49, widths=(12, 32, 32, 4096))
    for bad_ctx in (True, False):
        c, t = ctx.copy(), tgt.copy()
        if bad_ctx:
            c[17, 3] = 4096
        else:
            t[200] = 65535
        tr = T.Trainer(layers, "fp32", max_batch=256)
        tr.forward(_dev(c), _dev(t))
        torch.cuda.synchronize()
        assert tr.status() == _lib.DLIC_ERR_INVALID
        tr.close()
    tr = T.Trainer(layers, "fp32", max_batch=256)
    tr.forward(_dev(ctx), _dev(tgt))
    assert tr.status() == 0
    tr.close()


def test_12bit_trained_network_codes_fewer_bits(T, orc):
    # 300 split-BF16 steps on contexts of 12-bit phantoms, then the slice is
    # coded with the untrained and the trained FP32 networks: bitstreams
    # equal to the oracle's, decodes exact, fewer bits after training
    from paper_2207_05152_gb300 import model as M
    from paper_2207_05152_gb300.codec import Codec
    imgs = _images(51, n=4, size=(128, 128))
    ctx, tgt = T.sample_contexts(imgs, 8192 * 300, 52)
    layers = synth.xavier_mlp([12, 128, 128, 4096], 53)
    tr = T.Trainer(layers, "bf16x3", max_batch=8192)
    c, t = _dev(ctx), _dev(tgt)
    first = last = None
    for k in range(300):
        loss = tr.step(c[k * 8192:(k + 1) * 8192], t[k * 8192:(k + 1) * 8192])
        if k == 0:
            first = float(loss.item())
    last = float(loss.item())
    torch.cuda.synchronize()
    assert tr.status() == 0
    assert last < first - 1.0, (first, last)
    test = synth.phantom_image12(64, 64, 99)
    sizes = {}
    for name, blob in (("untrained", M.fp32_blob12(layers)), ("trained", tr.fp32_blob())):
        codec = Codec(blob)
        dev = torch.from_numpy(test.view(np.int16)).cuda()
        got = codec.encode_to_bytes([dev], [16])[0]
        assert got == orc.encode(blob, test, 16)
        dec, st = codec.decode_bytes([got])
        assert st == [0] and np.array_equal(dec[0].astype(np.uint16), test)
        sizes[name] = len(got)
        codec.close()
    tr.close()
    assert sizes["trained"] < 0.9 * sizes["untrained"], sizes
