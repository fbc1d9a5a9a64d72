"""GPU parity at the configured workloads' own sizes and weights.

Every bitstream the GPU writes is compared byte for byte with the oracle's
for the same seeded inputs, and every decode must reproduce its image
(Sec. II-B "Preprocessor": encoder and decoder compute the same PDFs, the
image is reproduced losslessly):
- cfg 1: one 64 x 64 value-noise image, FP32 12-64-64-256 with seeded
  Xavier weights (near-uniform tables), 32 streams;
- the 512 x 512 image with Xavier weights of widths 128 in both precisions
  (the tensor-core encoder and the cluster decoders on near-uniform tables);
- cfg 4: the whole batch of 64 uneven images (72.8 Mpixel), INT8, automatic
  stream counts and cluster sizes;
- cfg 5: the 128 MRI-like slices coded with the untrained (Xavier) INT8
  network and with the network after 2000 BF16 training steps.
The oracle runs one host thread per image (it is plain C, called through
ctypes, which releases the interpreter lock)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import synth
from paper_2207_05152_gb300 import model as M
from paper_2207_05152_gb300 import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def Codec():
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300.codec import Codec
    return Codec


def _oracle_bitstreams(orc, blob, imgs, streams):
    orc.lib()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(lambda a: orc.encode(blob, a[0], a[1]), zip(imgs, streams)))


def _parity(Codec, orc, blob, imgs, streams=None):
    from paper_2207_05152_gb300 import _lib
    codec = Codec(blob)
    dev = [torch.from_numpy(np.ascontiguousarray(i)).cuda() for i in imgs]
    got = codec.encode_to_bytes(dev, streams)
    S = streams or [_lib.dlic_auto_streams(*i.shape) for i in imgs]
    want = _oracle_bitstreams(orc, blob, imgs, S)
    bad = [k for k in range(len(imgs)) if got[k] != want[k]]
    assert not bad, f"bitstreams differ from the oracle for images {bad[:8]}"
    data = torch.frombuffer(bytearray(b"".join(got)), dtype=torch.uint8).cuda()
    offs = np.concatenate([[0], np.cumsum([len(b) for b in got])]).tolist()
    outs, status = codec.decode(data, offs, [i.shape for i in imgs])
    torch.cuda.synchronize()
    assert status[:len(imgs)].cpu().tolist() == [0] * len(imgs)
    assert all(torch.equal(a, b) for a, b in zip(outs, dev)), "decoded pixels differ from the images"
    codec.close()
    return got


def test_cfg1_xavier_fp32_64x64_s32(Codec, orc):
    img = synth.config_image(1)
    blob = M.fp32_blob(synth.xavier_mlp([12, 64, 64, 256], 1))
    got = _parity(Codec, orc, blob, [img], [32])
    # near-uniform tables: close to 8 bits per pixel
    assert 7.0 < 8.0 * len(got[0]) / img.size < 9.0


@pytest.mark.parametrize("prec", ["int8", "fp32"])
def test_xavier_512x512_s256(Codec, orc, prec):
    img = workloads.cfg2_image()
    layers = synth.xavier_mlp([12, 128, 128, 256], 2)
    blob = M.int8_blob(layers, workloads.calibration_contexts()) if prec == "int8" else M.fp32_blob(layers)
    _parity(Codec, orc, blob, [img], [256])


def test_cfg4_whole_batch(Codec, orc):
    imgs = workloads.cfg4_images(64)
    assert sum(i.size for i in imgs) == 72785176
    _, blob8, _ = workloads.models()
    _parity(Codec, orc, blob8, imgs)


def test_cfg5_untrained_and_trained(Codec, orc):
    imgs = workloads.cfg5_images(128)
    run = workloads.cfg5_training(2000, "bf16", 65536, images=imgs)
    assert run["status"] == 0
    sizes = {}
    for name in ("untrained", "trained"):
        blob = M.int8_blob(run[name], run["calib"])
        got = _parity(Codec, orc, blob, imgs)
        sizes[name] = sum(len(b) for b in got)
    # the trained network codes the slices in fewer bits (Sec. IV-D)
    assert sizes["trained"] < sizes["untrained"]
