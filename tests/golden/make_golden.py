"""Writes the regression fixtures tests/golden/*.hex with the oracle alone.

Each case is a tiny image (or volume), a model blob packed here with struct
(the model blob layout: "DLM1", u32 precision, n_in, h1, h2, 256, window
field, f32 tscale, u32 lut[64], then the layers) and a stream count.  The
window fields: 2 (the default 12 priors), 1 << 24 | u | l << 8 | r << 16
(Fig. 6's 9 x 9: u = 8, l = 6, r = 2, 78 priors), or for a 3D window
2 << 28 | u | l << 4 | r << 8 | pu << 10 | pd << 14 | pl << 18 | pr << 22.  The fixtures pin the
oracle's bitstream bytes against later edits: a change to them must name the
passage of the paper, or the reading of it, that justifies it.
Run: python tests/golden/make_golden.py
"""
import os
import struct
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def _blob_fp32(layers, h1, h2, n_in=12, field=2):
    lut = np.rint(np.exp2(23.0 - np.arange(64) / 64.0)).astype("<u4")
    out = b"DLM1" + struct.pack("<6If", 0, n_in, h1, h2, 256, field, float(np.float32(64.0 / np.log(2.0))))
    out += lut.tobytes()
    for w, b in layers:
        out += np.asarray(w, "<f4").tobytes() + np.asarray(b, "<f4").tobytes()
    return out


def cases():
    import synth
    out = []
    layers = synth.predictive_mlp([12, 32, 32, 256], 5)
    blob = _blob_fp32(layers, 32, 32)
    out.append(("pred_fp32_9x13_s3", blob, synth.value_noise_image(9, 13, 42), 3))
    out.append(("pred_fp32_6x20_s1", blob, synth.voronoi_image(6, 20, 43), 1))
    zero = [(np.zeros((32, 12)), np.zeros(32)), (np.zeros((32, 32)), np.zeros(32)),
            (np.zeros((256, 32)), np.zeros(256))]
    out.append(("flat_fp32_5x5_s5", _blob_fp32(zero, 32, 32), synth.voronoi_image(5, 5, 44), 5))
    fig6 = synth.predictive_mlp([78, 32, 32, 256], 6, window=(8, 6, 2))
    out.append(("fig6_fp32_11x14_s2", _blob_fp32(fig6, 32, 32, 78, (1 << 24) | 8 | (6 << 8) | (2 << 16)),
                synth.value_noise_image(11, 14, 45), 2))
    return out


def volume_cases():
    """3D window (2, 2, 2) + the 3 x 3 neighbourhood one slice down."""
    import synth
    window = (2, 2, 2, 1, 1, 1, 1)
    field = (2 << 28) | 2 | (2 << 4) | (2 << 8) | (1 << 10) | (1 << 14) | (1 << 18) | (1 << 22)
    layers = synth.predictive_mlp([21, 32, 32, 256], 7, window=window)
    return [("vol_fp32_3x6x9_s2", _blob_fp32(layers, 32, 32, 21, field), synth.phantom_volume(3, 6, 9, 46), 2)]


if __name__ == "__main__":
    import oracle
    for name, blob, img, S in cases():
        with open(os.path.join(HERE, name + ".hex"), "w") as fh:
            fh.write(oracle.encode(blob, img, S).hex() + "\n")
        print("wrote", name)
    for name, blob, vol, S in volume_cases():
        with open(os.path.join(HERE, name + ".hex"), "w") as fh:
            fh.write(oracle.encode_volume(blob, vol, S)[0].hex() + "\n")
        print("wrote", name)
