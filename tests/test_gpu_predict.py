"""dlic_predict: the model's per-pixel frequency-table entry (f | c << 16)
of each pixel's own value, without coding, against the oracle's tables bit
for bit (Sec. II-B: a PDF per pixel quantised to the coder's table; Eq. 1),
for the INT8 tensor-core, FP32, one-CTA, deeper-network and 12-bit kernels,
batches of ragged images and the 512 x 512 image; and the ideal code length
sum -log2(f / 2^16) against the oracle's float64 sum."""
import numpy as np
import pytest
import torch

import synth
from paper_2207_05152_gb300 import model as M
from paper_2207_05152_gb300 import workloads
from tests.helpers import calib_contexts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Codec():
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300.codec import Codec
    return Codec


def _check(Codec, orc, blob, imgs, dtype=torch.uint8):
    codec = Codec(blob)
    dev = [torch.from_numpy(np.ascontiguousarray(i).view(np.int16) if dtype == torch.int16 else i).cuda()
           for i in imgs]
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    out = codec.predict(dev, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = out.cpu().numpy().view(np.uint32)
    off = 0
    for img in imgs:
        want, bits = orc.symbol_tables(blob, img)
        n = img.size
        assert np.array_equal(got[off:off + n].reshape(img.shape), want)
        f = (got[off:off + n] & 0xFFFF).astype(np.float64)
        assert abs(float(-np.log2(f / 65536.0).sum()) - bits) <= 1e-6 * max(1.0, bits)
        off += n
    codec.close()


SHAPES = [(1, 1), (1, 9), (7, 1), (5, 64), (33, 17), (70, 130)]


@pytest.mark.parametrize("prec,widths", [("int8", [12, 128, 128, 256]), ("int8", [12, 32, 48, 256]),
                                         ("fp32", [12, 64, 64, 256]), ("fp32", [12, 32, 256, 256])])
def test_predict_matches_oracle_tables(Codec, orc, prec, widths):
    imgs = [synth.value_noise_image(h, w, 3 * h + w) for h, w in SHAPES]
    layers = synth.predictive_mlp(widths, 5)
    blob = M.int8_blob(layers, calib_contexts([synth.voronoi_image(40, 40, 2)])) if prec == "int8" else M.fp32_blob(layers)
    _check(Codec, orc, blob, imgs)


def test_predict_512x512(Codec, orc):
    _, blob8, _ = workloads.models()
    _check(Codec, orc, blob8, [workloads.cfg2_image()])


def test_predict_deep_and_12bit(Codec, orc):
    deep8, deep32 = workloads.deep_models()
    imgs = [synth.voronoi_image(30, 41, 6), synth.voronoi_image(9, 70, 7)]
    _check(Codec, orc, deep8, imgs)
    _check(Codec, orc, deep32, imgs)
    layers = synth.predictive_mlp([12, 32, 32, 4096], 3, sigma=96.0, levels=4096)
    imgs12 = [synth.phantom_image12(20, 31, 4), synth.phantom_image12(7, 40, 5)]
    _check(Codec, orc, M.fp32_blob12(layers), imgs12, torch.int16)
