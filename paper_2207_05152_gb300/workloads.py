"""Named synthetic workloads of the benchmark and the profiling runner.

cfg2: one 512 x 512 Voronoi image, INT8 (and FP32) network 12-128-128-256
      with synthetic predictive weights, 256 rANS streams.
cfg4: a batch of Voronoi images of uneven sizes (default 64, heights
      192..1536, widths 256..2048), the same INT8 network, automatic streams.
"""
from __future__ import annotations

import numpy as np

import synth
from . import model as M

WIDTHS = [12, 128, 128, 256]


def calibration_contexts(seed: int = 4242, count: int = 4096) -> np.ndarray:
    """Priors of `count` pixels of a separate synthetic image (zero-padded),
    the calibration data of the INT8 quantisation."""
    cal_img = synth.voronoi_image(256, 256, seed)
    rng = synth.Rng(seed + 1)
    rr = rng.integers(count, 0, 255)
    cc = rng.integers(count, 0, 255)
    pad = np.zeros((258, 260), np.uint8)
    pad[2:, 2:258] = cal_img
    return np.stack([np.concatenate([pad[r:r + 2, c:c + 5].reshape(-1), pad[r + 2, c:c + 2]])
                     for r, c in zip(rr, cc)])


def models(seed: int = 2):
    """(layers, INT8 blob, FP32 blob) of the synthetic predictive network."""
    layers = synth.predictive_mlp(WIDTHS, seed)
    return layers, M.int8_blob(layers, calibration_contexts()), M.fp32_blob(layers)


def cfg2_image() -> np.ndarray:
    return synth.config_image(2)


def cfg4_images(count: int = 64, seed: int = 4000, **size_kw):
    return synth.batch_images(count, seed, **size_kw)


def cfg5_images(count: int = 128, seed: int = 5000):
    """MRI-like slices: elliptical phantoms with a bias field and Rician noise."""
    import synth as _s
    return [_s.phantom_image(512, 512, seed + i) for i in range(count)]
