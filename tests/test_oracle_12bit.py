"""The oracle with 12-bit pixels (Sec. IV "Higher Bit Depth": one 12-bit
channel, a network of 4096 output neurons).

Pins:
- closed forms of the 4096-way table: equal logits give f_i = 16 for every
  value (2^16 / 4096), one dominant logit gives it 2^16 - 4095 and every
  other value 1;
- a bound on random logits: the table tracks 1 + 61440 softmax_i within
  the lut grid's error;
- the uniform network codes any 12-bit image at 12 bits per pixel plus
  the streams' flush words;
- the network's logits for 12-bit priors against float64 with inputs
  v / 2048 - 1;
- round trips over ragged shapes and stream counts; the container's 12-bit
  flag; refusals (INT8 with 4096 outputs, samples above 4095, an 8-bit model
  on a 12-bit stream)."""
import math
import struct

import numpy as np
import pytest

import synth
from paper_2207_05152_gb300 import model as M


def _lut():
    return M.table_lut()


def _zero_net(h=32):
    z = np.float32
    return [(np.zeros((h, 12), z), np.zeros(h, z)), (np.zeros((h, h), z), np.zeros(h, z)),
            (np.zeros((4096, h), z), np.zeros(4096, z))]


def test_equal_logits_give_sixteen_each(orc):
    cum = orc.table_from_logits(np.full(4096, 1.25, np.float32), M.TSCALE, _lut())
    assert cum.size == 4097
    assert np.array_equal(cum, 16 * np.arange(4097, dtype=np.uint32))


@pytest.mark.parametrize("s", [0, 1, 2047, 4095])
def test_one_dominant_logit(orc, s):
    z = np.full(4096, -1000.0, np.float32)
    z[s] = 3.0
    f = np.diff(orc.table_from_logits(z, M.TSCALE, _lut()).astype(np.int64))
    want = np.ones(4096, np.int64)
    want[s] = 65536 - 4095
    assert np.array_equal(f, want)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_table_tracks_the_softmax(orc, seed):
    rng = synth.Rng(seed)
    z = (3.0 * rng.normal(4096)).astype(np.float32)   # a spread of about 25 nats: no clamping
    cum = orc.table_from_logits(z, M.TSCALE, _lut()).astype(np.int64)
    f = np.diff(cum)
    assert cum[0] == 0 and cum[-1] == 65536 and f.min() >= 1
    p = np.exp(z.astype(np.float64) - z.max())
    p /= p.sum()
    # each weight is 2^23 exp(z - m) on a grid of 1/64 bit (relative error
    # <= 2^(1/128) - 1 from rounding u, and the floor of each cumulative
    # value moves f by less than 2 units)
    err = np.abs((f - 1) - 61440.0 * p)
    assert np.all(err <= 0.0055 * 61440.0 * p + 2.0)


def test_uniform_network_codes_twelve_bits_per_pixel(orc):
    blob = M.fp32_blob12(_zero_net())
    img = synth.phantom_image12(23, 41, 5)
    S = 5
    data = orc.encode(blob, img, S)
    words = struct.unpack_from(f"<{S}I", data, 24)
    assert len(data) == 24 + 4 * S + 2 * sum(words)
    # payload bits beyond the flush words against 12 bits per pixel: the
    # state carries at most 16 bits of each stream's last symbols
    payload_bits = 16 * (sum(words) - 2 * S)
    n = img.size
    assert 12 * n - 16 * S <= payload_bits <= 12 * n
    st, dec = orc.decode(blob, data, *img.shape)
    assert st == 0 and np.array_equal(dec, img)


def test_logits_against_float64(orc):
    layers = synth.predictive_mlp([12, 64, 64, 4096], 7, sigma=40.0, levels=4096)
    blob = M.fp32_blob12(layers)
    rng = synth.Rng(9)
    pri = rng.integers(300, 0, 4096).reshape(25, 12).astype(np.uint16)
    z = orc.logits(blob, pri)
    assert z.shape == (25, 4096)
    x = pri.astype(np.float64) / 2048.0 - 1.0
    for li, (w, b) in enumerate(layers):
        x = x @ w.astype(np.float64).T + b
        if li < 2:
            x = np.maximum(x, 0.0)
    assert np.max(np.abs(z - x)) <= 1e-5 * np.abs(x).max()


SHAPES = [(1, 1, 1), (7, 1, 4), (1, 9, 1), (5, 64, 3), (33, 17, 32), (20, 37, 7)]


@pytest.mark.parametrize("h,w,s", SHAPES)
def test_round_trip(orc, h, w, s):
    layers = synth.predictive_mlp([12, 32, 32, 4096], 3, sigma=96.0, levels=4096)
    blob = M.fp32_blob12(layers)
    img = synth.phantom_image12(h, w, 100 + h + w) if h > 1 and w > 1 else \
        synth.Rng(h * w).integers(h * w, 0, 4096).reshape(h, w).astype(np.uint16)
    data = orc.encode(blob, img, s)
    assert data[13] == 0x10                       # FP32, 12-bit pixels
    st, dec = orc.decode(blob, data, h, w)
    assert st == 0 and dec.dtype == np.uint16 and np.array_equal(dec, img)
    fc, bits = orc.symbol_tables(blob, img)
    payload = 16 * (sum(struct.unpack_from(f"<{min(s, h)}I", data, 24)) - 2 * min(s, h))
    assert payload <= bits + 16 * min(s, h) + 1e-6 * img.size
    assert math.isfinite(bits)


def test_refusals(orc):
    img = synth.phantom_image12(9, 11, 4)
    blob = M.fp32_blob12(synth.predictive_mlp([12, 32, 32, 4096], 3, sigma=96.0, levels=4096))
    bad = img.copy()
    bad[4, 5] = 4096                              # not a 12-bit value
    with pytest.raises(ValueError):
        orc.encode(blob, bad, 3)
    # an INT8 network with 4096 outputs (well-formed, sizes consistent) is
    # not a valid model: an INT8 input byte cannot hold a 12-bit prior
    i8 = [M._header(M.PREC_INT8, 32, 32, M.DEFAULT_WINDOW, 4096)]
    for o, i in ((32, 12), (32, 32), (4096, 32)):
        i8 += [np.zeros((o, i), np.int8).tobytes(), np.ones(o, "<f4").tobytes(), np.zeros(o, "<f4").tobytes()]
    with pytest.raises(ValueError):
        orc.encode(b"".join(i8), img, 3)
    # an 8-bit model does not decode a 12-bit stream (container flag, hash)
    data = orc.encode(blob, img, 3)
    b8 = M.fp32_blob(synth.predictive_mlp([12, 32, 32, 256], 3))
    st, _ = orc.decode(b8, data, 9, 11)
    assert st == 3
    flag = bytearray(data)
    flag[13] = 0                                  # the 12-bit flag cleared
    st, _ = orc.decode(blob, bytes(flag), 9, 11)
    assert st == 3


def test_deeper_12bit_network_in_the_dlm2_blob(orc):
    # three hidden layers and 4096 outputs: the "DLM2" header fields, float64
    # logits with inputs v / 2048 - 1, and a round trip
    rng = synth.Rng(17)
    dims = [12, 40, 24, 56, 4096]
    layers = [((rng.normal(o * i).reshape(o, i) * np.sqrt(2.0 / i)).astype(np.float32),
               (0.05 * rng.normal(o)).astype(np.float32)) for i, o in zip(dims[:-1], dims[1:])]
    blob = M.deep_fp32_blob(layers)
    assert blob[:4] == b"DLM2" and M.model_symbols(blob) == 4096 and orc.symbols(blob) == 4096
    prec, n_in, L = struct.unpack_from("<3I", blob, 4)
    widths = struct.unpack_from("<8I", blob, 16)
    assert (prec, n_in, L) == (0, 12, 3) and widths == (40, 24, 56, 0, 0, 0, 0, 0)
    assert struct.unpack_from("<I", blob, 48)[0] == 4096
    pri = synth.Rng(18).integers(60, 0, 4096).reshape(5, 12).astype(np.uint16)
    z = orc.logits(blob, pri)
    x = pri.astype(np.float64) / 2048.0 - 1.0
    for li, (w, b) in enumerate(layers):
        x = x @ w.astype(np.float64).T + b
        if li < len(layers) - 1:
            x = np.maximum(x, 0.0)
    assert np.max(np.abs(z - x)) <= 1e-5 * np.abs(x).max()
    img = synth.phantom_image12(14, 19, 2)
    data = orc.encode(blob, img, 3)
    st, dec = orc.decode(blob, data, 14, 19)
    assert st == 0 and np.array_equal(dec, img)
    with pytest.raises(ValueError):   # INT8 with 4096 outputs has no blob
        M.deep_int8_blob(layers, np.zeros((4, 12), np.uint8))


def test_twelve_bit_volume_round_trip(orc):
    # the paper's MRI setting: 12-bit slices with a 3D window (Sec. IV); a
    # model whose lower-layer weights are zero codes every slice like the 2D
    # model of the same other weights (the lower layer only adds zero terms)
    win3 = M.VOLUME_WINDOW
    n3 = M.window_size(win3)
    rng = synth.Rng(31)
    w1 = (rng.normal(32 * n3).reshape(32, n3) * 0.2).astype(np.float32)
    w1[:, 12:] = 0.0
    rest = [((rng.normal(32 * 32).reshape(32, 32) * 0.2).astype(np.float32), np.zeros(32, np.float32)),
            ((rng.normal(4096 * 32).reshape(4096, 32) * 0.2).astype(np.float32), np.zeros(4096, np.float32))]
    b1 = np.zeros(32, np.float32)
    blob3 = M.deep_fp32_blob([(w1, b1)] + rest, win3)
    blob2 = M.deep_fp32_blob([(np.ascontiguousarray(w1[:, :12]), b1)] + rest)
    vol = np.stack([synth.phantom_image12(11, 13, 40 + z) for z in range(3)])
    data, offs = orc.encode_volume(blob3, vol, 4)
    st, dec = orc.decode_volume(blob3, data, offs, 3, 11, 13)
    assert st == 0 and dec.dtype == np.uint16 and np.array_equal(dec, vol)
    for z in range(3):
        sl = data[offs[z]:offs[z + 1]]
        flat = orc.encode(blob2, vol[z], 4)
        assert sl[12] == 2 | 0x80 and sl[13] == 0x10
        assert sl[24:] == flat[24:]                 # the payload: identical
