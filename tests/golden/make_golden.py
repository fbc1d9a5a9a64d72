"""Writes the regression fixtures tests/golden/*.hex with the oracle alone.

Each case is a tiny image, a model blob packed here with struct (the model
blob layout: "DLM1", u32 precision, 12, h1, h2, 256, 2, f32 tscale,
u32 lut[64], then the layers) and a stream count.  The fixtures pin the
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


def _blob_fp32(layers, h1, h2):
    lut = np.rint(np.exp2(23.0 - np.arange(64) / 64.0)).astype("<u4")
    out = b"DLM1" + struct.pack("<6If", 0, 12, h1, h2, 256, 2, float(np.float32(64.0 / np.log(2.0))))
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
    return out


if __name__ == "__main__":
    import oracle
    for name, blob, img, S in cases():
        with open(os.path.join(HERE, name + ".hex"), "w") as fh:
            fh.write(oracle.encode(blob, img, S).hex() + "\n")
        print("wrote", name)
