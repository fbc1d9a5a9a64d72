"""Pins of the oracle's whole coder: gather, network, wavefront order,
streams, container, round trip and code length.

Sec. II-A: the window holds only already-decoded pixels and decoding repeats
the encoder's prediction exactly; Fig. 1 right: pixels outside the image are
dummy values; Sec. II-B: wavefront processing and one rANS stream per row at
most; Sec. III-A: the cross-entropy in bits tracks the achieved rate
(excluding header information)."""
import os
import struct

import numpy as np
import pytest

import synth
from paper_2207_05152_gb300 import model as M
from tests.helpers import fp32_model, int8_model, fma32, f32

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DR = [-2, -2, -2, -2, -2, -1, -1, -1, -1, -1, 0, 0]
DC = [-2, -1, 0, 1, 2, -2, -1, 0, 1, 2, -2, -1]


def test_fnv1a64_published_vectors(orc):
    # Test vectors of the FNV reference (Fowler, Noll, Vo).
    with open(os.path.join(GOLDEN, "fnv1a64_vectors.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            text, hexval = line.rstrip("\n").split("\t")
            text = "" if text == "<empty>" else text
            assert orc.fnv1a64(text.encode()) == int(hexval, 16)


def test_gather_matches_padded_slices(orc):
    img = synth.voronoi_image(9, 11, 5)
    pad = np.zeros((13, 15), np.uint8)
    pad[2:11, 2:13] = img
    for r in range(9):
        for c in range(11):
            win = pad[r:r + 3, c:c + 5]
            want = np.concatenate([win[0], win[1], win[2, :2]])
            assert np.array_equal(orc.gather(img, r, c), want)


@pytest.mark.parametrize("H,W", [(8, 8), (5, 3), (1, 9), (9, 1), (4, 2), (7, 13)])
def test_wavefront_schedule(H, W):
    # t = 3r + c: every in-image prior lies on an earlier wave, and for
    # W >= 3 t equals the longest dependency chain ending at the pixel
    # (so no smaller slope is valid for this window).
    depth = np.zeros((H, W), np.int64)
    for r in range(H):
        for c in range(W):
            best = -1
            for dr, dc in zip(DR, DC):
                y, x = r + dr, c + dc
                if 0 <= y < H and 0 <= x < W:
                    assert 3 * y + x < 3 * r + c
                    best = max(best, depth[y, x])
            depth[r, c] = best + 1
    t = 3 * np.arange(H)[:, None] + np.arange(W)[None, :]
    if W >= 3:
        assert np.array_equal(depth, t)
    assert np.all(depth <= t)


def _np_forward_fp32(layers, pri):
    x = pri.astype(np.float64) / 128.0 - 1.0
    for li, (w, b) in enumerate(layers):
        x = x @ w.astype(np.float64).T + b.astype(np.float64)
        if li < 2:
            x = np.maximum(x, 0.0)
    return x


@pytest.mark.parametrize("widths", [[12, 64, 64, 256], [12, 128, 128, 256], [12, 32, 48, 256]])
def test_fp32_network_vs_float64(orc, widths):
    layers, blob = fp32_model(widths, seed=4, kind="xavier")
    rng = synth.Rng(11)
    pri = rng.integers(64 * 12, 0, 255).reshape(64, 12).astype(np.uint8)
    z = orc.logits(blob, pri).astype(np.float64)
    ref = _np_forward_fp32(layers, pri)
    scale = np.abs(ref).max() + 1.0
    assert np.abs(z - ref).max() <= 2e-6 * scale * widths[1]


def test_fp32_network_exact_order(orc):
    # The first logit of a tiny case recomputed with exact fma emulation in
    # the stated order (bias first, k ascending).
    layers, blob = fp32_model([12, 16, 16, 256], seed=8, kind="xavier")
    pri = np.array([[0, 1, 2, 100, 200, 255, 7, 9, 128, 127, 50, 60]], np.uint8)
    a = [f32(v / 128.0 - 1.0) for v in pri[0]]
    for li, (w, b) in enumerate(layers):
        out = []
        for j in range(w.shape[0]):
            acc = float(b[j])
            for k in range(w.shape[1]):
                acc = fma32(a[k], float(w[j, k]), acc)
            out.append(max(acc, 0.0) if li < 2 else acc)
        a = out
    z = orc.logits(blob, pri)[0]
    assert np.array_equal(z.astype(np.float64), np.array(a))


def test_int8_network_exact(orc):
    images = [synth.voronoi_image(64, 64, 3)]
    layers, blob = int8_model([12, 32, 32, 256], images, seed=2)
    d = M.parse_blob(blob)
    rng = synth.Rng(12)
    pri = rng.integers(6 * 12, 0, 255).reshape(6, 12).astype(np.uint8)
    z = orc.logits(blob, pri)
    for n in range(pri.shape[0]):
        a = [int(v) - 128 for v in pri[n]]
        for li in (1, 2, 3):
            q, s, o = d[f"Q{li}"].astype(np.int64), d[f"s{li}"], d[f"o{li}"]
            acc = q @ np.array(a, np.int64)
            if li < 3:
                a = [int(min(max(np.rint(np.float32(fma32(float(acc[j]), float(s[j]), float(o[j])))), 0), 255))
                     for j in range(len(acc))]
            else:
                want = [fma32(float(acc[j]), float(s[j]), float(o[j])) for j in range(len(acc))]
        assert np.array_equal(z[n].astype(np.float64), np.array(want))


def test_int8_tracks_fp32(orc):
    images = [synth.voronoi_image(64, 64, 3)]
    layers, blob8 = int8_model([12, 64, 64, 256], images, seed=2)
    blob32 = M.fp32_blob(layers)
    img = images[0]
    _, b32 = orc.symbol_tables(blob32, img)
    _, b8 = orc.symbol_tables(blob8, img)
    assert abs(b32 - b8) / img.size < 0.05


SHAPES = [(1, 1, 1), (1, 7, 1), (7, 1, 4), (2, 3, 2), (5, 64, 9), (16, 16, 16), (13, 40, 3),
          (9, 50, 1), (33, 17, 32)]


@pytest.mark.parametrize("H,W,S", SHAPES)
@pytest.mark.parametrize("prec", ["fp32", "int8"])
def test_roundtrip_shapes(orc, H, W, S, prec):
    img = synth.value_noise_image(H, W, H * 100 + W)
    if prec == "fp32":
        _, blob = fp32_model([12, 32, 32, 256], seed=H + W)
    else:
        _, blob = int8_model([12, 32, 32, 256], [synth.voronoi_image(32, 32, 1)], seed=H + W)
    data = orc.encode(blob, img, S)
    st, dec = orc.decode(blob, data, H, W)
    assert st == 0
    assert np.array_equal(dec, img)
    Se = min(S, H)
    assert len(data) <= orc.max_encoded_bytes(H, W, S)
    assert data[:4] == b"DLC1"
    h, w, rad, prec_tag, s_hdr = struct.unpack_from("<IIBBH", data, 4)
    assert (h, w, rad, s_hdr) == (H, W, 2, Se)
    assert prec_tag == (0 if prec == "fp32" else 1)
    (hash_,) = struct.unpack_from("<Q", data, 16)
    assert hash_ == orc.fnv1a64(blob)
    words = struct.unpack_from(f"<{Se}I", data, 24)
    assert len(data) == 24 + 4 * Se + 2 * sum(words)


def _stream_symbols(img, S, s):
    H, W = img.shape
    px = [(3 * r + c, r, c) for r in range(s, H, S) for c in range(W)]
    return [int(img[r, c]) for _, r, c in sorted(px)]


@pytest.mark.parametrize("H,W,S", [(8, 8, 2), (12, 40, 3), (5, 5, 5), (30, 7, 1)])
def test_flat_tables_closed_form(orc, H, W, S):
    # Zero weights: every table is flat (f = 256, c = 256 s), so each rANS
    # step multiplies the state range by exactly 256.  Per stream, the
    # payload carries exactly 8 bits per symbol:
    #   16 * (renorm words) + floor(log2 x_final) - 16 == 8 n,
    # and the bytes follow the power-of-two form of the step:
    #   x >= 2^24 -> emit x mod 2^16, x >>= 16;  x = (x >> 8) << 16 | s << 8 | x & 255.
    layers = [(np.zeros((32, 12), np.float32), np.zeros(32, np.float32)),
              (np.zeros((32, 32), np.float32), np.zeros(32, np.float32)),
              (np.zeros((256, 32), np.float32), np.zeros(256, np.float32))]
    blob = M.fp32_blob(layers)
    img = synth.voronoi_image(H, W, 9)
    data = orc.encode(blob, img, S)
    words = struct.unpack_from(f"<{S}I", data, 24)
    pos = 24 + 4 * S
    for s in range(S):
        syms = _stream_symbols(img, S, s)
        x, emitted = 1 << 16, []
        for v in reversed(syms):
            if x >= 1 << 24:
                emitted.append(x & 0xFFFF)
                x >>= 16
            x = ((x >> 8) << 16) | (v << 8) | (x & 0xFF)
        want = [x >> 16, x & 0xFFFF] + emitted[::-1]
        got = list(struct.unpack_from(f"<{words[s]}H", data, pos))
        pos += 2 * words[s]
        assert got == want
        assert 16 * (words[s] - 2) + (x.bit_length() - 1) - 16 == 8 * len(syms)


def test_code_length_tracks_cross_entropy(orc):
    # Payload bits (excluding header and the 32-bit flush of each stream)
    # are within 0.01 bpp of the summed -log2(f / 2^16).
    img = synth.config_image(1)
    _, blob = fp32_model([12, 64, 64, 256], seed=3)
    S = 32
    data = orc.encode(blob, img, S)
    _, ideal = orc.symbol_tables(blob, img)
    words = struct.unpack_from(f"<{S}I", data, 24)
    pos = 24 + 4 * S
    bits = 0.0
    for s in range(S):
        hi, lo = struct.unpack_from("<HH", data, pos)
        x = (hi << 16) | lo
        bits += 16 * (words[s] - 2) + np.log2(x) - 16
        pos += 2 * words[s]
    assert abs(bits - ideal) / img.size <= 0.01
    assert ideal / img.size < 6.0   # the predictive weights give a peaked PDF


def test_corrupt_streams_are_rejected(orc):
    img = synth.value_noise_image(16, 24, 4)
    _, blob = fp32_model([12, 32, 32, 256], seed=1)
    data = bytearray(orc.encode(blob, img, 4))
    st, _ = orc.decode(blob, bytes(data[:-2]), 16, 24)
    assert st == 3
    st, _ = orc.decode(blob, bytes(data), 16, 25)
    assert st == 3
    other = fp32_model([12, 32, 32, 256], seed=2)[1]
    st, _ = orc.decode(other, bytes(data), 16, 24)
    assert st == 3
    bad = bytearray(data)
    bad[24 + 4 * 4] ^= 0x40            # first flush word of stream 0
    st, dec = orc.decode(blob, bytes(bad), 16, 24)
    assert st == 3 or not np.array_equal(dec, img)


def test_golden_small_bitstreams(orc):
    # Regression fixtures written by tests/golden/make_golden.py (oracle only).
    import importlib.util
    spec = importlib.util.spec_from_file_location("mg", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    for name, blob, img, S in mg.cases():
        with open(os.path.join(GOLDEN, name + ".hex")) as fh:
            want = bytes.fromhex(fh.read().strip())
        assert orc.encode(blob, img, S) == want, name
    for name, blob, vol, S in mg.volume_cases():
        with open(os.path.join(GOLDEN, name + ".hex")) as fh:
            want = bytes.fromhex(fh.read().strip())
        assert orc.encode_volume(blob, vol, S)[0] == want, name
