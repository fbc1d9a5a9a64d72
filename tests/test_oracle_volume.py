"""The oracle with 3D windows and volumes (Sec. IV "3D Dependencies": a
two-layer window, the lower layer from the previous slice and possibly
reaching below the target's row; "3D Wavefront": the 2D wavefronts of the
slices overlap, each slice shifted so that its lower-layer priors are already
decoded).

Pins: the 3D gather against slices of zero-padded arrays (the first slice's
lower layer is all zeros); the wave shift 3 pd + pr + 1 against brute force
(every prior on an earlier wave of T = 3r + c + shift z, and no smaller shift
works); a 3D model whose lower-layer weights are zero codes every slice with
the payload of the 2D model it extends; round trips of volumes on edge shapes
for both precisions; the slice header; 2D and volume calls refusing each
other's models."""
import numpy as np
import pytest

import synth
from paper_2207_05152_gb300 import model as M
from tests.helpers import calib_contexts

VOL = M.VOLUME_WINDOW
WINDOWS3 = [VOL, (1, 1, 1, 0, 0, 0, 0), (2, 3, 1, 2, 2, 2, 2), (3, 2, 2, 0, 3, 1, 4), (8, 6, 2, 1, 0, 0, 1)]


def _slices(window, below, img, y, x):
    u, l, r, pu, pd, pl, pr = window
    H, W = img.shape
    P = 10
    pad = np.zeros((H + 2 * P, W + 2 * P), np.uint8)
    pad[P:P + H, P:P + W] = img
    rows = [pad[P + y - d, P + x - l:P + x + r + 1] for d in range(u, 0, -1)]
    own = np.concatenate(rows + [pad[P + y, P + x - l:P + x]])
    if below is None:
        low = np.zeros((pu + pd + 1) * (pl + pr + 1), np.uint8)
    else:
        padb = np.zeros_like(pad)
        padb[P:P + H, P:P + W] = below
        low = padb[P + y - pu:P + y + pd + 1, P + x - pl:P + x + pr + 1].reshape(-1)
    return np.concatenate([own, low])


@pytest.mark.parametrize("window", WINDOWS3)
def test_gather3_matches_padded_slices(orc, window):
    vol = synth.phantom_volume(3, 13, 17, 4)
    for (y, x) in [(0, 0), (5, 7), (12, 16), (3, 0), (0, 16), (8, 2), (12, 0)]:
        for z in range(3):
            below = vol[z - 1] if z else None
            got = orc.gather_window3(window, below, vol[z], y, x)
            assert np.array_equal(got, _slices(window, below, vol[z], y, x)), (window, z, y, x)


@pytest.mark.parametrize("window", WINDOWS3)
def test_wave_shift_is_smallest_topological(window):
    # T(z, r, c) = 3r + c + shift z: every prior of a pixel, in its own slice
    # or the one before, lies on an earlier T; with shift - 1 one does not
    u, l, rr, pu, pd, pl, pr = window
    shift = M.volume_wave_shift(window)
    offs = M.window_offsets3(window)
    D, H, W = 3, 12, 14

    def ok(sh):
        for z in range(D):
            for r in range(H):
                for c in range(W):
                    T = 3 * r + c + sh * z
                    for dz, dr, dc in offs:
                        zz, y, x = z + dz, r + dr, c + dc
                        if 0 <= zz and 0 <= y < H and 0 <= x < W and 3 * y + x + sh * zz >= T:
                            return False
        return True

    assert ok(shift)
    assert not ok(shift - 1)


def _volume_models(widths, seed, vol, window, prec):
    layers = synth.predictive_mlp(widths, seed, window=window)
    if prec == "fp32":
        return M.fp32_blob(layers, window)
    return M.int8_blob(layers, calib_contexts(list(vol), window=window), window)


@pytest.mark.parametrize("prec", ["fp32", "int8"])
@pytest.mark.parametrize("D,H,W,S", [(1, 1, 1, 1), (2, 1, 9, 1), (3, 7, 1, 4), (4, 16, 23, 4), (5, 11, 30, 11)])
def test_volume_roundtrip(orc, prec, D, H, W, S):
    vol = synth.phantom_volume(D, H, W, 7 * D + H)
    blob = _volume_models([M.window_size(VOL), 32, 32, 256], 3, vol, VOL, prec)
    data, offs = orc.encode_volume(blob, vol, S)
    assert len(offs) == D + 1 and offs[0] == 0 and offs[-1] == len(data)
    for z in range(D):
        assert data[offs[z]:offs[z] + 4] == b"DLC1" and data[offs[z] + 12] == 0x80 | VOL[0]
    st, dec = orc.decode_volume(blob, data, offs, D, H, W)
    assert st == 0 and np.array_equal(dec, vol)


def test_zero_lower_layer_codes_like_2d(orc):
    # a 3D model whose lower-layer weights are zero predicts like the 2D
    # model it extends: every slice carries the 2D coder's payload
    vol = synth.phantom_volume(3, 20, 27, 9)
    l2 = synth.predictive_mlp([12, 32, 32, 256], 5)
    w1, b1 = l2[0]
    w1z = np.concatenate([w1, np.zeros((w1.shape[0], 9), np.float32)], axis=1)
    l3 = [(w1z, b1)] + l2[1:]
    b2d, b3d = M.fp32_blob(l2), M.fp32_blob(l3, VOL)
    data, offs = orc.encode_volume(b3d, vol, 5)
    for z in range(3):
        want = orc.encode(b2d, vol[z], 5)
        got = data[offs[z]:offs[z + 1]]
        assert got[24:] == want[24:] and got[:12] == want[:12] and got[13:16] == want[13:16]
    # and the lower layer does reach the tables when its weights are not zero
    l3n = [(w1z + np.float32(0.0), b1)] + l2[1:]
    l3n[0][0][:, 12 + 4] = 0.5
    data_n, offs_n = orc.encode_volume(M.fp32_blob(l3n, VOL), vol, 5)
    assert data_n[offs_n[1] + 24:offs_n[2]] != data[offs[1] + 24:offs[2]]


def test_volume_and_2d_calls_refuse_each_other(orc):
    vol = synth.phantom_volume(2, 9, 10, 1)
    b3d = _volume_models([M.window_size(VOL), 32, 32, 256], 3, vol, VOL, "fp32")
    b2d = M.fp32_blob(synth.predictive_mlp([12, 32, 32, 256], 3))
    with pytest.raises(ValueError):
        orc.encode(b3d, vol[0], 2)
    with pytest.raises(ValueError):
        orc.encode_volume(b2d, vol, 2)
    data, offs = orc.encode_volume(b3d, vol, 2)
    st, _ = orc.decode(b3d, data[:offs[1]], 9, 10)
    assert st != 0
    # a slice is bound to its volume's model (hash) and window byte
    st, _ = orc.decode_volume(b3d, data[:offs[1]] + data[offs[1]:], offs, 2, 9, 10)
    assert st == 0
    bad = bytearray(data)
    bad[offs[1] + 12] ^= 0x80
    st, _ = orc.decode_volume(b3d, bytes(bad), offs, 2, 9, 10)
    assert st == 3


def test_window_fields_round_trip():
    for w in WINDOWS3:
        assert M.window_of_field(M.window_field(w)) == w
    with pytest.raises(ValueError):
        M.window_field((2, 2, 3, 1, 1, 1, 1))
    with pytest.raises(ValueError):
        M.window_field((8, 8, 2, 2, 2, 2, 2))      # 148 priors


def test_blob_writer_matches_the_struct_layout():
    # the package's blob writer, for the 9 x 9 and the 3D window, against the
    # layout packed field by field in the golden-fixture script
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "make_golden.py")
    spec = importlib.util.spec_from_file_location("mg", path)
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    fig6 = synth.predictive_mlp([78, 32, 32, 256], 6, window=M.FIG6_WINDOW)
    assert M.fp32_blob(fig6, M.FIG6_WINDOW) == [c for c in mg.cases() if c[0].startswith("fig6")][0][1]
    vol = synth.predictive_mlp([21, 32, 32, 256], 7, window=VOL)
    assert M.fp32_blob(vol, VOL) == mg.volume_cases()[0][1]


@pytest.mark.parametrize("window", [VOL, (3, 2, 2, 0, 3, 1, 4)])
def test_training_contexts_match_the_oracle_gather(orc, window):
    # the trainer's context sampler over the slices of a volume gives, at
    # every sampled voxel, the oracle's 3D gather
    from paper_2207_05152_gb300 import train as T
    vol = synth.phantom_volume(4, 12, 15, 30)
    slices = list(vol)
    ctx, tgt = T.sample_window_contexts(slices, 300, 31, window)
    idx, rr, cc = synth.sample_positions(slices, 300, 31)
    for n, (z, r, c) in enumerate(zip(idx, rr, cc)):
        want = orc.gather_window3(window, slices[z - 1] if z else None, slices[z], int(r), int(c))
        assert np.array_equal(ctx[n], want), (z, r, c)
        assert tgt[n] == slices[z][r, c]
