"""GPU parity for 12-bit pixels (Sec. IV "Higher Bit Depth": one 12-bit
channel, 4096 output neurons): the warp-per-pixel FP32 encoder and decoder
against the oracle, bit for bit, on seeded MRI-like 12-bit slices of ragged
shapes, several stream counts, batches, pitched rows, networks of one, two
and three hidden layers, and corrupt streams."""
import numpy as np
import pytest
import torch

import synth
from paper_2207_05152_gb300 import model as M

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (7, 1, 4), (1, 9, 1), (5, 64, 3), (33, 17, 32), (20, 37, 7), (48, 70, 16)]


@pytest.fixture(scope="module")
def Codec():
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300.codec import Codec
    return Codec


def _image(h, w, seed):
    if h > 1 and w > 1:
        return synth.phantom_image12(h, w, seed)
    return synth.Rng(seed).integers(h * w, 0, 4096).reshape(h, w).astype(np.uint16)


def _dev(img):
    return torch.from_numpy(img.astype(np.int16)).cuda()


def _check(Codec, orc, blob, imgs, streams):
    codec = Codec(blob)
    got = codec.encode_to_bytes([_dev(i) for i in imgs], streams)
    for k, img in enumerate(imgs):
        assert got[k] == orc.encode(blob, img, streams[k]), f"image {k}: bitstream differs from the oracle"
    dec, status = codec.decode_bytes(got)
    assert status == [0] * len(imgs)
    for k, img in enumerate(imgs):
        assert dec[k].dtype == np.uint16 and np.array_equal(dec[k], img), f"image {k}: decode differs"
    codec.close()
    return got


def _blob12(hidden=(32, 32), seed=3, sigma=96.0):
    layers = synth.predictive_mlp([12, 32, 32, 4096], seed, sigma=sigma, levels=4096)
    if tuple(hidden) == (32, 32):
        return M.fp32_blob12(layers)
    rng = synth.Rng(seed + 100)
    dims = [12] + list(hidden) + [4096]
    deep = [((rng.normal(o * i).reshape(o, i) * np.sqrt(2.0 / i)).astype(np.float32),
             (0.05 * rng.normal(o)).astype(np.float32)) for i, o in zip(dims[:-1], dims[1:])]
    return M.deep_fp32_blob(deep)


def test_shapes_and_streams(Codec, orc):
    imgs = [_image(h, w, 7 * h + w) for h, w, _ in SHAPES]
    _check(Codec, orc, _blob12(), imgs, [s for _, _, s in SHAPES])


@pytest.mark.parametrize("hidden", [(64,), (48, 96, 32)])
def test_other_depths(Codec, orc, hidden):
    imgs = [_image(21, 30, 5), _image(9, 44, 6)]
    _check(Codec, orc, _blob12(hidden), imgs, [5, 9])


def test_wide_hidden_layers(Codec, orc):
    # hidden widths of 256: the kernels' largest activation buffers
    layers = synth.predictive_mlp([12, 256, 256, 4096], 4, sigma=64.0, levels=4096)
    img = _image(18, 26, 8)
    _check(Codec, orc, M.fp32_blob12(layers), [img], [6])


def test_pitched_rows(Codec, orc):
    blob = _blob12()
    img = _image(19, 23, 9)
    wide = torch.zeros((19, 40), dtype=torch.int16, device="cuda")
    wide[:, :23] = _dev(img)
    view = wide[:, :23]                            # pitch 80 bytes
    codec = Codec(blob)
    got = codec.encode_to_bytes([view], [4])[0]
    assert got == orc.encode(blob, img, 4)
    out = torch.full((19, 40), -1, dtype=torch.int16, device="cuda")
    data = torch.frombuffer(bytearray(got), dtype=torch.uint8).cuda()
    outs, status = codec.decode(data, [0, len(got)], [(19, 23)], outs=[out[:, :23]])
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    host = out.cpu().numpy()
    assert np.array_equal(host[:, :23].view(np.uint16), img) and np.all(host[:, 23:] == -1)
    codec.close()


def test_corrupt_stream_is_reported(Codec, orc):
    from paper_2207_05152_gb300 import _lib
    blob = _blob12()
    img = _image(20, 30, 2)
    codec = Codec(blob)
    data = bytearray(orc.encode(blob, img, 4))
    _, st = codec.decode_bytes([bytes(data[:-2])], [(20, 30)])
    assert st == [_lib.DLIC_ERR_CORRUPT]
    bad = bytearray(data)
    bad[13] = 0                                    # the 12-bit flag cleared
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


@pytest.mark.parametrize("value", [4096, 65535])
def test_samples_above_4095_are_refused(Codec, orc, value):
    # a 12-bit sample beyond the 4096-value table has no frequency: the
    # oracle refuses the image, and the device writes DLIC_ERR_INVALID to
    # the encode status word
    from paper_2207_05152_gb300 import _lib
    blob = _blob12()
    img = _image(17, 29, 4)
    img[9, 13] = value
    with pytest.raises(ValueError):
        orc.encode(blob, img, 4)
    codec = Codec(blob)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    codec.encode([torch.from_numpy(img.view(np.int16)).cuda()], [4], status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == _lib.DLIC_ERR_INVALID
    # the same call on a valid image afterwards reports success
    img[9, 13] = 4095
    status.zero_()
    codec.encode([_dev(img)], [4], status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    codec.close()
