"""The oracle with other causal windows ("any window shape", Sec. II-A; the
9 x 9 window of Fig. 6 with the target in the last row, third column from the
right: rows r-8..r-1 at columns c-6..c+2, then row r at columns c-6..c-1).

Pins: the gather against padded slicing; the default window against the
12-prior gather; the wavefront t = 3r + c still being a topological order and,
for the Fig. 6 window, the exact longest-path depth; the network against
float64 and exact-integer arithmetic; round trips; the container's window byte;
malformed windows rejected."""
import numpy as np
import pytest

import synth
from paper_2207_05152_gb300 import model as M
from tests.helpers import calib_contexts, window_offsets

FIG6 = M.FIG6_WINDOW
WINDOWS = [(2, 2, 2), FIG6, (1, 3, 1), (4, 1, 2), (3, 0, 2)]


@pytest.mark.parametrize("window", WINDOWS)
def test_gather_matches_padded_slices(orc, window):
    u, l, r = window
    img = synth.value_noise_image(13, 17, 3)
    pad = np.zeros((13 + u, 17 + l + r), np.uint8)
    pad[u:, l:l + 17] = img
    for (y, x) in [(0, 0), (5, 7), (12, 16), (3, 0), (0, 16), (8, 2)]:
        got = orc.gather_window(window, img, y, x)
        rows = [pad[y + u - d, x:x + l + r + 1] for d in range(u, 0, -1)]
        want = np.concatenate(rows + [pad[y + u, x:x + l]])
        assert np.array_equal(got, want), (window, y, x)
    if window == (2, 2, 2):
        for (y, x) in [(0, 0), (5, 7), (12, 16)]:
            assert np.array_equal(orc.gather_window(window, img, y, x), orc.gather(img, y, x))


@pytest.mark.parametrize("window", WINDOWS)
def test_wavefront_is_topological(window):
    # every in-image prior of (r, c) lies on an earlier wave of t = 3r + c
    # (a right reach of at most 2); for the Fig. 6 window the longest
    # dependency chain ending at a pixel is exactly 3r + c
    H, W = 14, 19
    depth = np.zeros((H, W), np.int64)
    offs = window_offsets(window)
    for r in range(H):
        for c in range(W):
            best = -1
            for dr, dc in offs:
                y, x = r + dr, c + dc
                if 0 <= y < H and 0 <= x < W:
                    assert 3 * y + x < 3 * r + c
                    best = max(best, depth[y, x])
            depth[r, c] = best + 1
    t = 3 * np.arange(H)[:, None] + np.arange(W)[None, :]
    assert np.all(depth <= t)
    if window[2] == 2 and window[1] >= 1:
        assert np.array_equal(depth, t)


def _fp64_forward(layers, pri):
    x = pri.astype(np.float64) / 128.0 - 1.0
    for li, (w, b) in enumerate(layers):
        x = x @ w.astype(np.float64).T + b.astype(np.float64)
        if li < 2:
            x = np.maximum(x, 0.0)
    return x


def test_fig6_fp32_network_vs_float64(orc):
    layers = synth.predictive_mlp([78, 64, 64, 256], 3, window=FIG6)
    blob = M.fp32_blob(layers, FIG6)
    rng = synth.Rng(5)
    pri = rng.integers(200 * 78, 0, 255).astype(np.uint8).reshape(200, 78)
    z = orc.logits(blob, pri)
    want = _fp64_forward(layers, pri)
    assert np.max(np.abs(z - want)) <= 1e-4 * max(1.0, np.abs(want).max())


def test_fig6_int8_network_exact(orc):
    img = synth.voronoi_image(40, 40, 2)
    layers = synth.predictive_mlp([78, 64, 64, 256], 3, window=FIG6)
    blob = M.int8_blob(layers, calib_contexts([img], window=FIG6), FIG6)
    d = M.parse_blob(blob)
    assert d["n_in"] == 78 and d["window"] == FIG6
    rng = synth.Rng(6)
    pri = rng.integers(50 * 78, 0, 255).astype(np.uint8).reshape(50, 78)
    z = orc.logits(blob, pri)
    a = pri.astype(np.int64) - 128
    for li in range(3):
        acc = a @ d[f"Q{li + 1}"].astype(np.int64).T
        s, o = d[f"s{li + 1}"], d[f"o{li + 1}"]
        if li < 2:
            a = np.clip(np.rint(np.float32(acc.astype(np.float32)) * s + o), 0, 255).astype(np.int64)
            # fma(acc, s, o) rounds once; compare the float64 of the same
            # product-sum, which agrees except at exact halves
            exact = np.clip(np.rint(acc.astype(np.float64) * s.astype(np.float64) + o.astype(np.float64)), 0, 255)
            assert np.mean(a == exact) > 0.999
            a = exact.astype(np.int64)
        else:
            want = acc.astype(np.float64) * s.astype(np.float64) + o.astype(np.float64)
    assert np.max(np.abs(z - want)) <= 1e-5 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("prec", ["fp32", "int8"])
@pytest.mark.parametrize("H,W,S", [(1, 1, 1), (9, 1, 3), (1, 20, 1), (16, 23, 4), (30, 45, 30), (11, 64, 2)])
def test_fig6_roundtrip(orc, prec, H, W, S):
    img = synth.value_noise_image(H, W, 7 * H + W)
    layers = synth.predictive_mlp([78, 64, 64, 256], 4, window=FIG6)
    blob = (M.fp32_blob(layers, FIG6) if prec == "fp32"
            else M.int8_blob(layers, calib_contexts([synth.voronoi_image(40, 40, 2)], window=FIG6), FIG6))
    data = orc.encode(blob, img, S)
    assert data[12] == 8                      # rows of the window above the pixel
    st, dec = orc.decode(blob, data, H, W)
    assert st == 0 and np.array_equal(dec, img)
    bad = bytearray(data)
    bad[12] = 2
    st, _ = orc.decode(blob, bytes(bad), H, W)
    assert st != 0


def test_window_field_and_invalid_windows(orc):
    assert M.window_field((2, 2, 2)) == 2
    assert M.window_field(FIG6) == (1 << 24) | 8 | (6 << 8) | (2 << 16)
    assert M.window_of_field(M.window_field((3, 1, 0))) == (3, 1, 0)
    for bad in [(9, 2, 2), (2, 2, 3), (0, 2, 2), (8, 9, 2)]:   # rows, right reach, no rows, left reach
        with pytest.raises(ValueError):
            M.window_field(bad)
    # a blob whose window field says 3 rows but n_in says 12 is rejected
    layers = synth.predictive_mlp([12, 32, 32, 256], 1)
    blob = bytearray(M.fp32_blob(layers))
    blob[24:28] = ((1 << 24) | 3 | (2 << 8) | (2 << 16)).to_bytes(4, "little")
    with pytest.raises(ValueError):
        orc.encode(bytes(blob), synth.value_noise_image(4, 4, 1), 1)
