"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module draws random numbers and shapes them into the workloads the coder
is exercised on: 8-bit grayscale images with the structure of the paper's
photographs and MRI slices (Sec. III-A, Sec. IV-A), FP32 weights for the
12 -> h1 -> h2 -> 256 density-estimation network (Sec. II-B, "Neural Network
Architecture"), and (context, target) training pairs.  It holds none of the
coding method's arithmetic: no gather, no network evaluation, no table
quantisation, no entropy coding.  Both the CUDA path and the CPU oracle take
its outputs as plain inputs.

Randomness: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator, so value i
of stream `seed` is mix(seed * 2^32 + i + 1).  Gaussians use the Box-Muller
transform in float64.  Pixel values are rounded half-to-even and clamped to
0..255.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Values offset..offset+n-1 of SplitMix64 stream `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        base = np.uint64((int(seed) * (1 << 32)) & 0xFFFFFFFFFFFFFFFF)
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = (base + ctr) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Rng:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """Doubles in [lo, hi) from the top 53 bits."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        """Standard normal deviates by Box-Muller (cosine branch only)."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers in [lo, hi] (inclusive), by scaling a uniform double."""
        u = self.uniform(n)
        return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def _to_u8(a: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(a), 0, 255).astype(np.uint8)


def _smoothstep(t: np.ndarray) -> np.ndarray:
    return t * t * (3.0 - 2.0 * t)


def value_noise_image(height: int, width: int, seed: int, sigma: float = 4.0) -> np.ndarray:
    """Smooth "Perlin-like" field plus N(0, sigma^2): 4 octaves of value noise
    on lattices of 8, 16, 32 and 64 pixels with smoothstep interpolation,
    rescaled to 0..255, then noise added, rounded and clamped."""
    rng = Rng(seed)
    ys = np.arange(height, dtype=np.float64)[:, None]
    xs = np.arange(width, dtype=np.float64)[None, :]
    field = np.zeros((height, width))
    amp = 1.0
    for cell in (64, 32, 16, 8):
        gh, gw = height // cell + 2, width // cell + 2
        lat = rng.uniform(gh * gw).reshape(gh, gw)
        gy, gx = ys / cell, xs / cell
        iy, ix = np.floor(gy).astype(int), np.floor(gx).astype(int)
        ty, tx = _smoothstep(gy - iy), _smoothstep(gx - ix)
        a = lat[iy, ix]
        b = lat[iy, ix + 1]
        c = lat[iy + 1, ix]
        d = lat[iy + 1, ix + 1]
        field += amp * ((a * (1 - tx) + b * tx) * (1 - ty) + (c * (1 - tx) + d * tx) * ty)
        amp *= 0.5
    lo, hi = field.min(), field.max()
    field = (field - lo) / max(hi - lo, 1e-12) * 255.0
    field += sigma * rng.normal(height * width).reshape(height, width)
    return _to_u8(field)


def voronoi_image(height: int, width: int, seed: int, cells: int = 24) -> np.ndarray:
    """Piecewise-smooth image: `cells` Voronoi regions, each a random linear
    ramp (edges at the region borders), plus Gaussian noise whose sigma is
    drawn per region from U[2, 8]."""
    rng = Rng(seed)
    cy = rng.uniform(cells, 0, height)
    cx = rng.uniform(cells, 0, width)
    base = rng.uniform(cells, 20, 235)
    gy = rng.uniform(cells, -0.6, 0.6)
    gx = rng.uniform(cells, -0.6, 0.6)
    sig = rng.uniform(cells, 2.0, 8.0)
    ys = np.arange(height, dtype=np.float64)[:, None]
    xs = np.arange(width, dtype=np.float64)[None, :]
    best = np.full((height, width), np.inf)
    label = np.zeros((height, width), dtype=np.int64)
    for k in range(cells):
        d = (ys - cy[k]) ** 2 + (xs - cx[k]) ** 2
        m = d < best
        best[m] = d[m]
        label[m] = k
    img = base[label] + gy[label] * (ys - cy[label]) + gx[label] * (xs - cx[label])
    img += sig[label] * rng.normal(height * width).reshape(height, width)
    return _to_u8(img)


def phantom_image(height: int, width: int, seed: int) -> np.ndarray:
    """MRI-like slice: 3..8 nested ellipses of random centre, axes, angle and
    intensity, times a smooth quadratic bias field in [0.8, 1.2], with Rician
    noise sqrt((s + n1)^2 + n2^2), sigma drawn from U[3, 10]."""
    rng = Rng(seed)
    n_ell = int(rng.integers(1, 3, 8)[0])
    ys = (np.arange(height, dtype=np.float64)[:, None] - height / 2) / (height / 2)
    xs = (np.arange(width, dtype=np.float64)[None, :] - width / 2) / (width / 2)
    img = np.zeros((height, width))
    scale = 1.0
    for _ in range(n_ell):
        p = rng.uniform(6)
        y0, x0 = (p[0] - 0.5) * 0.3 * scale, (p[1] - 0.5) * 0.3 * scale
        ay, ax = (0.5 + 0.4 * p[2]) * scale, (0.5 + 0.4 * p[3]) * scale
        th = np.pi * p[4]
        val = 30.0 + 180.0 * p[5]
        yr = (ys - y0) * np.cos(th) + (xs - x0) * np.sin(th)
        xr = -(ys - y0) * np.sin(th) + (xs - x0) * np.cos(th)
        inside = (yr / ay) ** 2 + (xr / ax) ** 2 <= 1.0
        img[inside] = val
        scale *= 0.8
    q = rng.uniform(5, -0.1, 0.1)
    bias = 1.0 + q[0] * ys + q[1] * xs + q[2] * ys * ys + q[3] * xs * xs + q[4] * xs * ys
    bias = np.clip(bias, 0.8, 1.2)
    sigma = float(rng.uniform(1, 3.0, 10.0)[0])
    s = img * bias
    n1 = sigma * rng.normal(height * width).reshape(height, width)
    n2 = sigma * rng.normal(height * width).reshape(height, width)
    return _to_u8(np.sqrt((s + n1) ** 2 + n2 ** 2))


def phantom_image12(height: int, width: int, seed: int) -> np.ndarray:
    """12-bit MRI-like slice (uint16, 0..4095; Sec. IV: one 12-bit channel):
    the construction of phantom_image on a 16x finer intensity scale (tissue
    480..3360, Rician noise sigma from U[48, 160]), so that the background
    near zero dominates the histogram as in the paper's MRI data."""
    rng = Rng(seed)
    n_ell = int(rng.integers(1, 3, 8)[0])
    ys = (np.arange(height, dtype=np.float64)[:, None] - height / 2) / (height / 2)
    xs = (np.arange(width, dtype=np.float64)[None, :] - width / 2) / (width / 2)
    img = np.zeros((height, width))
    scale = 1.0
    for _ in range(n_ell):
        p = rng.uniform(6)
        y0, x0 = (p[0] - 0.5) * 0.3 * scale, (p[1] - 0.5) * 0.3 * scale
        ay, ax = (0.5 + 0.4 * p[2]) * scale, (0.5 + 0.4 * p[3]) * scale
        th = np.pi * p[4]
        val = 16.0 * (30.0 + 180.0 * p[5])
        yr = (ys - y0) * np.cos(th) + (xs - x0) * np.sin(th)
        xr = -(ys - y0) * np.sin(th) + (xs - x0) * np.cos(th)
        img[(yr / ay) ** 2 + (xr / ax) ** 2 <= 1.0] = val
        scale *= 0.8
    q = rng.uniform(5, -0.1, 0.1)
    bias = np.clip(1.0 + q[0] * ys + q[1] * xs + q[2] * ys * ys + q[3] * xs * xs + q[4] * xs * ys, 0.8, 1.2)
    sigma = 16.0 * float(rng.uniform(1, 3.0, 10.0)[0])
    s = img * bias
    n1 = sigma * rng.normal(height * width).reshape(height, width)
    n2 = sigma * rng.normal(height * width).reshape(height, width)
    return np.clip(np.rint(np.sqrt((s + n1) ** 2 + n2 ** 2)), 0, 4095).astype(np.uint16)


def phantom_volume(depth: int, height: int, width: int, seed: int) -> np.ndarray:
    """MRI-like volume (depth x height x width): 3..8 nested ellipsoids of
    random centre, axes, in-plane angle and intensity, times a smooth
    quadratic bias field in [0.8, 1.2], with Rician noise
    sqrt((s + n1)^2 + n2^2), sigma drawn from U[3, 10]; consecutive slices
    share the anatomy, as the slices of a scan do."""
    rng = Rng(seed)
    n_ell = int(rng.integers(1, 3, 8)[0])
    zs = (np.arange(depth, dtype=np.float64)[:, None, None] - depth / 2) / max(depth / 2, 1.0)
    ys = (np.arange(height, dtype=np.float64)[None, :, None] - height / 2) / (height / 2)
    xs = (np.arange(width, dtype=np.float64)[None, None, :] - width / 2) / (width / 2)
    vol = np.zeros((depth, height, width))
    scale = 1.0
    for _ in range(n_ell):
        p = rng.uniform(8)
        z0, y0, x0 = (p[0] - 0.5) * 0.3 * scale, (p[1] - 0.5) * 0.3 * scale, (p[2] - 0.5) * 0.3 * scale
        az, ay, ax = (0.8 + 0.6 * p[3]) * scale, (0.5 + 0.4 * p[4]) * scale, (0.5 + 0.4 * p[5]) * scale
        th = np.pi * p[6]
        val = 30.0 + 180.0 * p[7]
        yr = (ys - y0) * np.cos(th) + (xs - x0) * np.sin(th)
        xr = -(ys - y0) * np.sin(th) + (xs - x0) * np.cos(th)
        inside = (yr / ay) ** 2 + (xr / ax) ** 2 + ((zs - z0) / az) ** 2 <= 1.0
        vol[inside] = val
        scale *= 0.8
    q = rng.uniform(6, -0.1, 0.1)
    bias = np.clip(1.0 + q[0] * ys + q[1] * xs + q[2] * zs + q[3] * ys * ys + q[4] * xs * xs + q[5] * zs * zs,
                   0.8, 1.2)
    sigma = float(rng.uniform(1, 3.0, 10.0)[0])
    s = vol * bias
    n1 = sigma * rng.normal(s.size).reshape(s.shape)
    n2 = sigma * rng.normal(s.size).reshape(s.shape)
    return _to_u8(np.sqrt((s + n1) ** 2 + n2 ** 2))


def uneven_sizes(count: int, seed: int, hmin=192, hmax=1536, wmin=256, wmax=2048):
    """Heights and widths drawn independently and uniformly (inclusive)."""
    rng = Rng(seed)
    hs = rng.integers(count, hmin, hmax)
    ws = rng.integers(count, wmin, wmax)
    return [(int(h), int(w)) for h, w in zip(hs, ws)]


def xavier_mlp(widths, seed: int):
    """FP32 weights of a dense network with the given layer widths
    (e.g. [12, 64, 64, 256]).  W_l has shape (out, in) and is drawn from
    U(-a, a) with a = sqrt(6 / (in + out)) (Glorot and Bengio 2010); biases
    are zero.  Returns [(W1, b1), (W2, b2), ...] as float32 arrays."""
    rng = Rng(seed)
    layers = []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        w = rng.uniform(fan_in * fan_out, -a, a).reshape(fan_out, fan_in).astype(np.float32)
        layers.append((w, np.zeros(fan_out, dtype=np.float32)))
    return layers


def sample_positions(images, count: int, seed: int):
    """`count` (image, row, col) triples drawn uniformly over all pixels of
    the given list of images (pixel-weighted)."""
    rng = Rng(seed)
    sizes = np.array([im.shape[0] * im.shape[1] for im in images], dtype=np.int64)
    cum = np.concatenate([[0], np.cumsum(sizes)])
    flat = np.floor(rng.uniform(count) * cum[-1]).astype(np.int64)
    img = np.searchsorted(cum, flat, side="right") - 1
    rem = flat - cum[img]
    widths = np.array([im.shape[1] for im in images], dtype=np.int64)
    return img, rem // widths[img], rem % widths[img]


def config_image(cfg: int, index: int = 0) -> np.ndarray:
    """The synthetic image of workload `cfg` (1, 2 or 5) with the given index;
    seed = 1000 * cfg + index."""
    seed = 1000 * cfg + index
    if cfg == 1:
        return value_noise_image(64, 64, seed, sigma=4.0)
    if cfg in (2, 3):
        return voronoi_image(512, 512, seed)
    if cfg == 5:
        return phantom_image(512, 512, seed)
    raise ValueError(cfg)


def batch_images(count: int, seed: int, **size_kw):
    """`count` Voronoi images of uneven sizes (the batched-coding workload)."""
    sizes = uneven_sizes(count, seed, **size_kw)
    return [voronoi_image(h, w, seed * 131 + i + 1) for i, (h, w) in enumerate(sizes)]


def predictive_mlp(widths, seed: int, sigma: float = 6.0, noise: float = 0.02, window=(2, 2, 2), levels: int = 256):
    """FP32 weights for which the network's PDF is a discretised Gaussian of
    standard deviation `sigma` grey levels around a linear prediction from the
    priors (the mean of the left and upper neighbours plus a gradient term),
    plus small seeded perturbations in every weight.  The prediction is
    carried through the ReLU layers as relu(x) - relu(-x), so the network
    represents it exactly; it gives realistic, peaked tables without a
    training run.  Input features are v / 128 - 1 in the prior order of the
    causal window (u, l, r): rows r-u..r-1 at columns c-l..c+r, then row r at
    columns c-l..c-1 (the default (2, 2, 2): r-2: c-2..c+2, r-1: c-2..c+2,
    r: c-2, c-1), then for a 3D window (u, l, r, pu, pd, pl, pr) the
    previous slice's rows r-pu..r+pd at columns c-pl..c+pr.  With the
    default window every prior is carried through the ReLU layers, otherwise
    the ones that the prediction uses (for a 3D window also the previous
    slice's pixel at the target's position)."""
    u, l, rr = window[:3]
    wid = l + rr + 1
    n2 = u * wid + l
    n = n2
    i_left, i_up, i_upleft = u * wid + l - 1, (u - 1) * wid + l, (u - 1) * wid + l - 1
    carried = list(range(n)) if tuple(window) == (2, 2, 2) else [i_upleft, i_up, i_left]
    if len(window) == 7:
        # 3D window: the previous slice's pixel at the target's position joins
        pu, pd, pl, pr = window[3:]
        n += (pu + pd + 1) * (pl + pr + 1)
        i_below = n2 + pu * (pl + pr + 1) + pl
        carried = [i_upleft, i_up, i_left, i_below]
    n_in, h1, h2, n_out = widths
    nc = 2 * len(carried)
    assert n_in == n and n_out == levels and h1 >= nc and h2 >= nc and l >= 1
    rng = Rng(seed)
    alpha = np.zeros(n)
    alpha[i_left] = 0.75      # left neighbour
    alpha[i_up] = 0.75        # upper neighbour
    alpha[i_upleft] = -0.5    # upper-left neighbour
    if len(window) == 7:
        alpha[:n2] *= 0.75
        alpha[i_below] = 0.25     # the same position one slice down
    w1 = noise * rng.normal(h1 * n).reshape(h1, n)
    w1[:nc] = 0.0
    for j, k in enumerate(carried):
        w1[2 * j, k] = 1.0
        w1[2 * j + 1, k] = -1.0
    b1 = np.zeros(h1)
    w2 = noise * rng.normal(h2 * h1).reshape(h2, h1) / np.sqrt(h1)
    w2[:nc, :] = 0.0
    w2[:nc, :nc] = np.eye(nc)
    b2 = np.zeros(h2)
    half = levels / 2.0   # inputs and output levels as v / half - 1
    t = np.arange(levels) / half - 1.0
    beta = 1.0 / (2.0 * (sigma / half) ** 2)
    pred = np.zeros(h2)
    for j, k in enumerate(carried):
        pred[2 * j] = alpha[k]
        pred[2 * j + 1] = -alpha[k]
    w3 = 2.0 * beta * t[:, None] * pred[None, :]
    w3 += noise * rng.normal(levels * h2).reshape(levels, h2)
    b3 = -beta * t * t
    return [(w1.astype(np.float32), b1.astype(np.float32)),
            (w2.astype(np.float32), b2.astype(np.float32)),
            (w3.astype(np.float32), b3.astype(np.float32))]
