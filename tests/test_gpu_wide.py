"""GPU parity for networks with hidden layers wider than 256 (Sec. II-B
"Neural Network Architecture": 128 to 4096 neurons per hidden layer): the
layer-at-a-time encoder and wave-at-a-time decoder, bit for bit against the
oracle on the same seeded inputs, in FP32 and INT8.

Networks: two hidden layers of 320 and 512 (a "DLM1"-shaped network too
wide for the fixed-depth kernels), three hidden layers of mixed widths up to
1024, and one hidden layer of 4096 (the widest of the paper) on small images.
Shapes span single pixels, ragged tails of the 4096-pixel passes and stream
counts below the wave length (streams shared by rows of one wave)."""
import numpy as np
import pytest
import torch

import synth
from paper_2207_05152_gb300 import model as M
from tests.helpers import calib_contexts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Codec():
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300.codec import Codec
    return Codec


def _random_layers(widths, seed):
    rng = synth.Rng(seed)
    layers, n = [], widths[0]
    for o in widths[1:]:
        w = (rng.normal(o * n).reshape(o, n) * np.sqrt(2.0 / n)).astype(np.float32)
        b = (0.05 * rng.normal(o)).astype(np.float32)
        layers.append((w, b))
        n = o
    return layers


def _blob(layers, prec, imgs):
    return M.deep_fp32_blob(layers) if prec == "fp32" else M.deep_int8_blob(layers, calib_contexts(imgs))


def _check(Codec, orc, blob, imgs, streams):
    codec = Codec(blob)
    got = codec.encode_to_bytes([torch.from_numpy(np.ascontiguousarray(i)).cuda() for i in imgs], streams)
    for k, img in enumerate(imgs):
        assert got[k] == orc.encode(blob, img, streams[k]), f"image {k}: bitstream differs from the oracle"
    dec, status = codec.decode_bytes(got)
    assert status == [0] * len(imgs)
    for k, img in enumerate(imgs):
        assert np.array_equal(dec[k], img), f"image {k}: decode differs from the input"
    codec.close()
    return got


SHAPES = [(1, 1, 1), (7, 1, 4), (1, 9, 1), (5, 64, 3), (33, 17, 2), (40, 71, 5), (70, 61, 70)]


@pytest.mark.parametrize("prec", ["fp32", "int8"])
@pytest.mark.parametrize("widths", [[12, 320, 512, 256], [12, 1024, 260, 300, 256]])
def test_wide_hidden_layers(Codec, orc, prec, widths):
    imgs = [synth.value_noise_image(h, w, 13 * h + w) for h, w, _ in SHAPES]
    streams = [s for _, _, s in SHAPES]
    _check(Codec, orc, _blob(_random_layers(widths, 31), prec, imgs[-2:]), imgs, streams)


@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_predictive_network_widened(Codec, orc, prec):
    # the predictive network with a hidden identity layer of 512 units: the
    # extra units carry zeros, so the tables are those of the 3-layer network
    base = synth.predictive_mlp([12, 64, 64, 256], 9)
    (w1, b1), (w2, b2), (w3, b3) = base
    wide = np.zeros((512, 64), np.float32)
    wide[:64] = np.eye(64, dtype=np.float32)
    w3w = np.zeros((256, 512), np.float32)
    w3w[:, :64] = w3
    layers = [(w1, b1), (w2, b2), (wide, np.zeros(512, np.float32)), (w3w, b3)]
    img = synth.voronoi_image(48, 80, 5)
    got = _check(Codec, orc, _blob(layers, prec, [img]), [img], [16])
    assert 8.0 * len(got[0]) / img.size < 7.0   # peaked tables, not near-uniform ones


@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_4096_wide_layer(Codec, orc, prec):
    imgs = [synth.value_noise_image(9, 11, 5), synth.value_noise_image(4, 30, 6)]
    _check(Codec, orc, _blob(_random_layers([12, 4096, 256], 33), prec, imgs), imgs, [3, 4])


def test_more_pixels_than_one_pass(Codec, orc):
    # 96 x 100 pixels: the encoder's passes (4096 pixels, 8192 on the tensor
    # cores) end mid-image
    img = synth.value_noise_image(96, 100, 7)
    _check(Codec, orc, _blob(_random_layers([12, 288, 256], 35), "int8", [img]), [img], [34])


def test_wide_corrupt_streams(Codec, orc):
    from paper_2207_05152_gb300 import _lib
    img = synth.value_noise_image(20, 30, 9)
    blob = _blob(_random_layers([12, 300, 256], 37), "fp32", [img])
    codec = Codec(blob)
    bits = codec.encode_to_bytes([torch.from_numpy(img).cuda()], [5])[0]
    bad = bytearray(bits)
    bad[-7] ^= 0x5A                       # a payload word
    short = bits[:-6]                     # a truncated container
    for data in (bytes(bad), short):
        _, st = codec.decode_bytes([data], shapes=[img.shape])
        want = orc.decode(blob, data, *img.shape)[0]
        assert (st[0] != 0) == (want != 0)
        if want:
            assert st[0] == _lib.DLIC_ERR_CORRUPT
    codec.close()
