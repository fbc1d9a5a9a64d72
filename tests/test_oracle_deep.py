"""The oracle with deeper networks (Sec. II-B "Neural Network Architecture":
six dense layers): the "DLM2" blob with 1..8 hidden layers of any widths.

Pins: hidden identity layers (W = I, b = 0 after a ReLU layer; exact in the
fixed fma order and, quantised, exact after requantisation) code every image
with the payload of the shallower network; a deep FP32 network's logits
against float64 and a deep INT8 network's against exact integer emulation;
round trips; malformed blobs refused."""
import struct

import numpy as np
import pytest

import synth
from paper_2207_05152_gb300 import model as M
from tests.helpers import calib_contexts


def _with_identities(layers, extra):
    """Insert `extra` identity hidden layers before the output layer."""
    h = layers[-2][0].shape[0]
    eye = [(np.eye(h, dtype=np.float32), np.zeros(h, np.float32)) for _ in range(extra)]
    return layers[:-1] + eye + layers[-1:]


def _random_deep(widths, seed):
    rng = synth.Rng(seed)
    layers, n = [], widths[0]
    for o in widths[1:]:
        w = (rng.normal(o * n).reshape(o, n) * np.sqrt(2.0 / n)).astype(np.float32)
        b = (0.05 * rng.normal(o)).astype(np.float32)
        layers.append((w, b))
        n = o
    return layers


@pytest.mark.parametrize("prec", ["fp32", "int8"])
@pytest.mark.parametrize("extra", [1, 3])
def test_identity_layers_code_like_the_shallow_network(orc, prec, extra):
    img = synth.voronoi_image(24, 37, 8)
    shallow = synth.predictive_mlp([12, 64, 64, 256], 9)
    deep = _with_identities(shallow, extra)
    if prec == "fp32":
        b3, bd = M.fp32_blob(shallow), M.deep_fp32_blob(deep)
    else:
        cal = calib_contexts([img])
        b3, bd = M.int8_blob(shallow, cal), M.deep_int8_blob(deep, cal)
    want, got = orc.encode(b3, img, 4), orc.encode(bd, img, 4)
    assert got[24:] == want[24:] and got[:16] == want[:16]   # all but the model hash
    st, dec = orc.decode(bd, got, 24, 37)
    assert st == 0 and np.array_equal(dec, img)


@pytest.mark.parametrize("widths", [[12, 64, 96, 48, 32, 80, 256],    # five hidden layers: six dense layers
                                    [12, 1024, 320, 256],             # hidden layers wider than 256
                                    [12, 4096, 256]])                 # the widest of Sec. II-B
def test_deep_fp32_logits_against_float64(orc, widths):
    layers = _random_deep(widths, 21)
    blob = M.deep_fp32_blob(layers)
    pri = synth.voronoi_image(16, 16, 3).reshape(-1, 1)[:, [0] * 12] ^ np.arange(12, dtype=np.uint8)
    z = orc.logits(blob, pri)
    x = pri.astype(np.float64) / 128.0 - 1.0
    for li, (w, b) in enumerate(layers):
        x = x @ w.astype(np.float64).T + b
        if li < len(layers) - 1:
            x = np.maximum(x, 0.0)
    assert np.max(np.abs(z - x)) <= 1e-4 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("widths", [[12, 48, 32, 64, 40, 256], [12, 1024, 2048, 256]])
def test_deep_int8_logits_exact(orc, widths):
    layers = _random_deep(widths, 23)
    img = synth.voronoi_image(30, 30, 4)
    cal = calib_contexts([img])
    blob = M.deep_int8_blob(layers, cal)
    pri = cal[:200]
    z = orc.logits(blob, pri)
    q = M._quantise(layers, cal)
    a = pri.astype(np.int64) - 128
    f32 = np.float32
    for li, (wq, s, o) in enumerate(q):
        acc = a @ wq.astype(np.int64).T
        s32, o32 = s.astype(f32), o.astype(f32)
        # fma(float(acc), s, o): the integer rounded to float32 first (exact
        # below 2^24; wide layers reach past it), then float64 holds the
        # product with s exactly; the float64 sum rounded to float32 differs
        # from a single rounding only on an exact float32 midpoint, which
        # these fixed inputs do not hit
        accf = acc.astype(f32).astype(np.float64)
        v = (accf * s32.astype(np.float64) + o32.astype(np.float64)).astype(f32)
        if li < len(q) - 1:
            a = np.clip(np.rint(v), 0, 255).astype(np.int64)
        else:
            assert np.array_equal(z, v)


@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_deep_roundtrips(orc, prec):
    layers = _with_identities(synth.predictive_mlp([12, 32, 32, 256], 5), 2)
    for H, W, S in [(1, 1, 1), (9, 1, 3), (13, 29, 4), (20, 45, 20)]:
        img = synth.value_noise_image(H, W, 3 * H + W)
        blob = M.deep_fp32_blob(layers) if prec == "fp32" else M.deep_int8_blob(layers, calib_contexts([img]))
        data = orc.encode(blob, img, S)
        st, dec = orc.decode(blob, data, H, W)
        assert st == 0 and np.array_equal(dec, img)


def test_malformed_deep_blobs(orc):
    layers = _with_identities(synth.predictive_mlp([12, 32, 32, 256], 5), 1)
    blob = bytearray(M.deep_fp32_blob(layers))
    img = synth.voronoi_image(5, 5, 1)
    orc.encode(bytes(blob), img, 1)
    for off, val in [(12, 0), (12, 9), (16 + 4 * 3, 32), (48, 255)]:
        bad = bytearray(blob)
        bad[off:off + 4] = struct.pack("<I", val)
        with pytest.raises(ValueError):
            orc.encode(bytes(bad), img, 1)
    with pytest.raises(ValueError):
        orc.encode(bytes(blob[:-4]), img, 1)
