"""Named synthetic workloads of the benchmark and the profiling runner.

cfg2: one 512 x 512 Voronoi image, INT8 (and FP32) network 12-128-128-256
      with synthetic predictive weights, 256 rANS streams.
volume: a 35 x 256 x 256 phantom scan (Table III's size) with the 3D window
      (2, 2, 2) + the 3 x 3 neighbourhood one slice down, 21-128-128-256.
fig6: the cfg2 image and streams with the 9 x 9 causal window of Fig. 6
      (78 priors), network 78-128-128-256.
cfg4: a batch of Voronoi images of uneven sizes (default 64, heights
      192..1536, widths 256..2048), the same INT8 network, automatic streams.
"""
from __future__ import annotations

import numpy as np

import synth
from . import model as M

WIDTHS = [12, 128, 128, 256]


def calibration_contexts(seed: int = 4242, count: int = 4096, window=M.DEFAULT_WINDOW) -> np.ndarray:
    """Priors of `count` pixels of a separate synthetic image (0 outside
    it), the calibration data of the INT8 quantisation; for a 3D window, of
    voxels of a separate synthetic volume."""
    if M.is_volume(window):
        return _volume_calibration(seed, count, window)
    cal_img = synth.voronoi_image(256, 256, seed)
    rng = synth.Rng(seed + 1)
    rr = rng.integers(count, 0, 255)
    cc = rng.integers(count, 0, 255)
    offs = M.window_offsets(window)
    out = np.zeros((count, len(offs)), np.uint8)
    for n, (r, c) in enumerate(zip(rr, cc)):
        for k, (dr, dc) in enumerate(offs):
            y, x = int(r) + dr, int(c) + dc
            if 0 <= y < 256 and 0 <= x < 256:
                out[n, k] = cal_img[y, x]
    return out


def _volume_calibration(seed: int, count: int, window) -> np.ndarray:
    cal = synth.phantom_volume(8, 128, 128, seed)
    rng = synth.Rng(seed + 1)
    zz = rng.integers(count, 0, 7)
    rr = rng.integers(count, 0, 127)
    cc = rng.integers(count, 0, 127)
    offs = M.window_offsets3(window)
    out = np.zeros((count, len(offs)), np.uint8)
    for n, (z, r, c) in enumerate(zip(zz, rr, cc)):
        for k, (dz, dr, dc) in enumerate(offs):
            v, y, x = int(z) + dz, int(r) + dr, int(c) + dc
            if v >= 0 and 0 <= y < 128 and 0 <= x < 128:
                out[n, k] = cal[v, y, x]
    return out


def volume_scan(depth: int = 35, size: int = 256, seed: int = 5100) -> np.ndarray:
    """A synthetic scan of `depth` slices of size x size (the 256 x 256 x 35
    of the paper's Table III by default)."""
    return synth.phantom_volume(depth, size, size, seed)


def models(seed: int = 2, window=M.DEFAULT_WINDOW, hidden: int = 128):
    """(layers, INT8 blob, FP32 blob) of the synthetic predictive network
    over the causal window (u, l, r)."""
    layers = synth.predictive_mlp([M.window_size(window), hidden, hidden, 256], seed, window=window)
    return (layers, M.int8_blob(layers, calibration_contexts(window=window), window),
            M.fp32_blob(layers, window))


def deep_models(seed: int = 2, extra: int = 3, hidden: int = 128):
    """(INT8 blob, FP32 blob) of a network of six dense layers (Sec. II-B):
    the synthetic predictive network with `extra` hidden identity layers
    (W = I, b = 0) before its output layer, as "DLM2" blobs."""
    layers = synth.predictive_mlp([M.window_size(M.DEFAULT_WINDOW), hidden, hidden, 256], seed)
    eye = [(np.eye(hidden, dtype=np.float32), np.zeros(hidden, np.float32)) for _ in range(extra)]
    deep = layers[:-1] + eye + layers[-1:]
    return M.deep_int8_blob(deep, calibration_contexts()), M.deep_fp32_blob(deep)


def wide_models(seed: int = 2, hidden: int = 4096):
    """(INT8 blob, FP32 blob) of a network with two hidden layers of `hidden`
    units (Sec. II-B: up to 4096 per hidden layer): the synthetic predictive
    network 12-64-64-256 in the first 64 units of each hidden layer, the
    other units with seeded random weights that the output layer does not
    read (its weights from them are zero), so the tables are realistic and
    every multiply-add of the dense layers is still done."""
    (w1, b1), (w2, b2), (w3, b3) = synth.predictive_mlp([M.window_size(M.DEFAULT_WINDOW), 64, 64, 256], seed)
    rng = synth.Rng(seed + 4096)
    n = w1.shape[1]
    W1 = (rng.normal(hidden * n).reshape(hidden, n) * np.sqrt(2.0 / n)).astype(np.float32)
    W1[:64] = w1
    B1 = (0.05 * rng.normal(hidden)).astype(np.float32)
    B1[:64] = b1
    W2 = (rng.normal(hidden * hidden).reshape(hidden, hidden) * np.sqrt(2.0 / hidden)).astype(np.float32)
    W2[:64, :] = 0.0
    W2[:64, :64] = w2
    B2 = (0.05 * rng.normal(hidden)).astype(np.float32)
    B2[:64] = b2
    W3 = np.zeros((256, hidden), np.float32)
    W3[:, :64] = w3
    layers = [(W1, B1), (W2, B2), (W3, b3.astype(np.float32))]
    return M.deep_int8_blob(layers, calibration_contexts()), M.deep_fp32_blob(layers)


def cfg2_image() -> np.ndarray:
    return synth.config_image(2)


def cfg4_images(count: int = 64, seed: int = 4000, **size_kw):
    return synth.batch_images(count, seed, **size_kw)


def cfg5_images(count: int = 128, seed: int = 5000):
    """MRI-like slices: elliptical phantoms with a bias field and Rician noise."""
    import synth as _s
    return [_s.phantom_image(512, 512, seed + i) for i in range(count)]


def cfg5_training(steps: int = 2000, mode: str = "bf16", batch: int = 65536, seed: int = 5000,
                  images=None):
    """cfg 5's training run on the current CUDA device: a 12-128-128-256
    network from seeded Xavier weights, `steps` steps of `batch` contexts
    drawn (on the device, seeded) from 2M contexts sampled uniformly from
    the 128 MRI-like slices.  Returns a dict with the untrained and trained
    layers, the calibration contexts of their INT8 quantisation (the first
    4096 sampled contexts), the final loss in bits and the seconds the
    steps took."""
    import time
    import torch
    from . import train as T
    imgs = images if images is not None else cfg5_images(128, seed)
    pool_ctx, pool_tgt = T.sample_contexts(imgs, 1 << 21, seed + 1)
    pc, pt = torch.from_numpy(pool_ctx).cuda(), torch.from_numpy(pool_tgt).cuda()
    layers0 = synth.xavier_mlp(WIDTHS, 5)
    tr = T.Trainer(layers0, mode, max_batch=batch)
    gen = torch.Generator(device="cuda").manual_seed(seed + 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        idx = torch.randint(0, pc.shape[0], (batch,), device="cuda", generator=gen)
        tr.step(pc.index_select(0, idx).contiguous(), pt.index_select(0, idx).contiguous())
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    status = tr.status()
    out = {"untrained": layers0, "trained": tr.layers(), "calib": pool_ctx[:4096],
           "final_loss_bits": float(tr.loss.item()), "seconds": seconds, "status": status}
    tr.close()
    return out
