"""GPU parity for networks of other than two hidden layers (Sec. II-B
"Neural Network Architecture": six dense layers): the "DLM2" blob on the
one-pixel-per-thread CUDA-core encoder, the cluster wavefront decoder's
warp-level MMA chain (INT8, 1..5 hidden layers of widths up to 128) and the
unit-split CUDA-core decoder (the rest), bit for bit against the oracle on
the same seeded inputs.

Networks: a predictive two-hidden-layer network with hidden identity layers
inserted (realistic, peaked tables), seeded random networks of five hidden
layers (six dense layers) of mixed widths, and a single hidden layer; every
network in FP32 and in INT8.  Image shapes span single pixels, ragged tails
of the 64-pixel prediction tiles and several stream counts."""
import numpy as np
import pytest
import torch

import synth
from paper_2207_05152_gb300 import model as M
from tests.helpers import calib_contexts

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (7, 1, 4), (1, 9, 1), (5, 64, 3), (33, 17, 32), (40, 71, 5), (64, 130, 16)]


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


def _with_identities(layers, extra):
    h = layers[-2][0].shape[0]
    eye = [(np.eye(h, dtype=np.float32), np.zeros(h, np.float32)) for _ in range(extra)]
    return layers[:-1] + eye + layers[-1:]


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


def _images():
    return [synth.value_noise_image(h, w, 11 * h + w) for h, w, _ in SHAPES], [s for _, _, s in SHAPES]


@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_identity_layers(Codec, orc, prec):
    # four hidden layers: the predictive network's two and two identities
    imgs, streams = _images()
    layers = _with_identities(synth.predictive_mlp([12, 64, 64, 256], 9), 2)
    _check(Codec, orc, _blob(layers, prec, imgs[-2:]), imgs, streams)


@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_six_dense_layers(Codec, orc, prec):
    imgs, streams = _images()
    layers = _random_layers([12, 64, 96, 48, 32, 80, 256], 21)
    _check(Codec, orc, _blob(layers, prec, imgs[-2:]), imgs, streams)


@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_widest_and_deepest(Codec, orc, prec):
    # eight hidden layers, widths up to 256 (the kernels' shared-memory maximum)
    imgs = [synth.voronoi_image(20, 37, 3), synth.value_noise_image(9, 70, 4)]
    layers = _random_layers([12, 256, 4, 128, 256, 36, 200, 16, 256, 256], 31)
    _check(Codec, orc, _blob(layers, prec, imgs), imgs, [3, 9])


@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_one_hidden_layer(Codec, orc, prec):
    imgs, streams = _images()
    layers = _random_layers([12, 64, 256], 41)
    _check(Codec, orc, _blob(layers, prec, imgs[-2:]), imgs, streams)


@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_two_hidden_layers_in_either_format(Codec, orc, prec):
    # a "DLM2" blob of two hidden layers runs the fixed-depth kernels and codes
    # every image like the same network as a "DLM1" blob (all but the hash)
    img = synth.config_image(1)
    layers = synth.predictive_mlp([12, 128, 128, 256], 2)
    cal = calib_contexts([img])
    b1 = M.fp32_blob(layers) if prec == "fp32" else M.int8_blob(layers, cal)
    b2 = M.deep_fp32_blob(layers) if prec == "fp32" else M.deep_int8_blob(layers, cal)
    g1 = _check(Codec, orc, b1, [img], [32])[0]
    g2 = _check(Codec, orc, b2, [img], [32])[0]
    assert g1[:16] == g2[:16] and g1[24:] == g2[24:] and g1[16:24] != g2[16:24]


def test_width_128_on_clusters(Codec, orc):
    # six dense layers of 128 units on images large enough for clusters of
    # several CTAs and waves of several pixel chunks per CTA, in one call
    imgs = [synth.voronoi_image(192, 256, 12), synth.value_noise_image(40, 400, 13), synth.value_noise_image(3, 700, 14)]
    layers = _random_layers([12, 128, 128, 128, 128, 128, 256], 61)
    _check(Codec, orc, _blob(layers, "int8", imgs), imgs, [64, 40, 3])


def test_predictive_six_layers(Codec, orc):
    # the bench's six-layer network (the predictive network with three
    # identity layers) on a 128 x 160 crop of the bench image: peaked tables
    from paper_2207_05152_gb300 import workloads
    img = np.ascontiguousarray(workloads.cfg2_image()[:128, :160])
    got = _check(Codec, orc, workloads.deep_models()[0], [img], [32])
    assert 8.0 * len(got[0]) / img.size < 7.0


def test_corrupt_stream_is_reported(Codec, orc):
    from paper_2207_05152_gb300 import _lib
    img = synth.value_noise_image(20, 30, 2)
    layers = _random_layers([12, 32, 48, 32, 256], 51)
    blob = _blob(layers, "int8", [img])
    codec = Codec(blob)
    data = bytearray(orc.encode(blob, img, 4))
    _, st = codec.decode_bytes([bytes(data[:-2])], [(20, 30)])
    assert st == [_lib.DLIC_ERR_CORRUPT]
    bad = bytearray(data)
    bad[16] ^= 1                                   # model hash
    _, st = codec.decode_bytes([bytes(bad)], [(20, 30)])
    assert st == [_lib.DLIC_ERR_CORRUPT]
    bad = bytearray(data)
    bad[24 + 16] ^= 0x80                           # first flush word of stream 0
    dec, st = codec.decode_bytes([bytes(bad)], [(20, 30)])
    want_status, want_img = orc.decode(blob, bytes(bad), 20, 30)
    assert (st[0] == 0) == (want_status == 0)
    if st[0] == 0:
        assert np.array_equal(dec[0], want_img)
    codec.close()
