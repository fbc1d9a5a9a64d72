"""Shared test helpers: model factories and exact reference arithmetic."""
from __future__ import annotations

import struct
from fractions import Fraction

import numpy as np

import synth
from paper_2207_05152_gb300 import model as M


def fp32_model(widths, seed=1, kind="predictive"):
    layers = synth.predictive_mlp(widths, seed) if kind == "predictive" else synth.xavier_mlp(widths, seed)
    return layers, M.fp32_blob(layers)


def window_offsets(window=(2, 2, 2)):
    """(dr, dc) of every prior of the causal window (u, l, r), in order."""
    u, l, r = window
    offs = [(-u + k // (l + r + 1), -l + k % (l + r + 1)) for k in range(u * (l + r + 1))]
    return offs + [(0, -l + k) for k in range(l)]


def calib_contexts(images, count=4096, seed=77, window=(2, 2, 2)):
    """Priors (u8 [count, window size]) of pixels drawn uniformly from the
    images, zero-padded at the borders: calibration data for quantisation.
    For a 3D window the images are the consecutive slices of a volume and
    the lower layer comes from the slice before (zeros for the first)."""
    idx, rr, cc = synth.sample_positions(images, count, seed)
    offs = [(0, dr, dc) for dr, dc in window_offsets(window[:3])]
    if len(window) == 7:
        pu, pd, pl, pr = window[3:]
        offs += [(-1, dr, dc) for dr in range(-pu, pd + 1) for dc in range(-pl, pr + 1)]
    out = np.zeros((count, len(offs)), np.uint8)
    for n, (i, r, c) in enumerate(zip(idx, rr, cc)):
        for k, (dz, dr, dc) in enumerate(offs):
            if i + dz < 0:
                continue
            img = images[i + dz]
            H, W = img.shape
            y, x = r + dr, c + dc
            out[n, k] = img[y, x] if 0 <= y < H and 0 <= x < W else 0
    return out


def int8_model(widths, images, seed=1):
    layers = synth.predictive_mlp(widths, seed)
    return layers, M.int8_blob(layers, calib_contexts(images))


def f32(x) -> float:
    return float(np.float32(x))


def round_to_f32(q: Fraction) -> float:
    """Correctly rounded (nearest, ties to even) float32 of an exact rational."""
    c = np.float32(float(q))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        d = abs(Fraction(float(cand)) - q)
        if best is None or d < best[0] or (d == best[0] and _even(cand) and not _even(best[1])):
            best = (d, cand)
    return float(best[1])


def _even(x) -> bool:
    return (struct.unpack("<I", struct.pack("<f", float(x)))[0] & 1) == 0


def fma32(a: float, b: float, c: float) -> float:
    """fma in float32: a*b+c exactly, rounded once."""
    return round_to_f32(Fraction(a) * Fraction(b) + Fraction(c))
