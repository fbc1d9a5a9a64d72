"""Rare-value upsampling of the training contexts (Sec. IV "Color
Frequencies": rare pixel values upsampled into the training set, the loss
weighted by value frequency).  Host-side sampling: checked against the
distributions it must draw from, and the contexts against the oracle's
gather."""
import numpy as np

import synth
from paper_2207_05152_gb300 import train as T


def _skewed_images():
    # MRI-like slices: a dark background dominates the value histogram
    return [synth.phantom_image(40, 56, 3), synth.phantom_image(33, 47, 4)]


def _chi2(counts, expected):
    m = expected > 0
    return float(np.sum((counts[m] - expected[m]) ** 2 / expected[m]))


def test_share_zero_is_the_uniform_sampler():
    imgs = _skewed_images()
    a = T.sample_upsampled_contexts(imgs, 3000, 11, share=0.0)
    b = T.sample_window_contexts(imgs, 3000, 11, (2, 2, 2))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_alpha_one_draws_every_present_value_equally():
    imgs = _skewed_images()
    n = 60000
    idx, rr, cc = T.rare_value_positions(imgs, n, 5, alpha=1.0)
    vals = np.array([imgs[i][r, c] for i, r, c in zip(idx, rr, cc)])
    present = np.unique(np.concatenate([im.reshape(-1) for im in imgs]))
    counts = np.bincount(vals, minlength=256)[present].astype(np.float64)
    k = present.size
    expected = np.full(k, n / k)
    # chi-square with k - 1 degrees of freedom: mean k - 1, sd sqrt(2 (k - 1))
    assert _chi2(counts, expected) < (k - 1) + 6.0 * np.sqrt(2.0 * (k - 1))
    assert np.all(counts > 0)


def test_alpha_zero_is_the_pixel_histogram():
    imgs = _skewed_images()
    n = 60000
    idx, rr, cc = T.rare_value_positions(imgs, n, 6, alpha=0.0)
    vals = np.array([imgs[i][r, c] for i, r, c in zip(idx, rr, cc)])
    flat = np.concatenate([im.reshape(-1) for im in imgs])
    hist = np.bincount(flat, minlength=256).astype(np.float64)
    counts = np.bincount(vals, minlength=256).astype(np.float64)
    expected = n * hist / hist.sum()
    k = int(np.count_nonzero(hist))
    assert _chi2(counts, expected) < (k - 1) + 6.0 * np.sqrt(2.0 * (k - 1))


def test_upsampling_raises_the_share_of_rare_values():
    imgs = _skewed_images()
    flat = np.concatenate([im.reshape(-1) for im in imgs])
    hist = np.bincount(flat, minlength=256)
    rare = hist[flat] <= np.percentile(hist[flat], 10)   # the pixels of the rarest values
    rare_share = rare.mean()
    _, tgt = T.sample_upsampled_contexts(imgs, 20000, 7, share=0.5)
    got = np.mean(hist[tgt] <= np.percentile(hist[flat], 10))
    assert got > 3.0 * rare_share


def test_contexts_match_the_oracle_gather(orc):
    imgs = _skewed_images()
    ctx, tgt = T.sample_upsampled_contexts(imgs, 400, 9, share=1.0)
    idx, rr, cc = T.rare_value_positions(imgs, 400, 9 + 0x5EED, 1.0)
    for k in range(0, 400, 37):
        img = imgs[idx[k]]
        assert tgt[k] == img[rr[k], cc[k]]
        assert np.array_equal(ctx[k], orc.gather(img, int(rr[k]), int(cc[k])))


def test_seeded():
    imgs = _skewed_images()
    a = T.sample_upsampled_contexts(imgs, 1000, 3)
    b = T.sample_upsampled_contexts(imgs, 1000, 3)
    c = T.sample_upsampled_contexts(imgs, 1000, 4)
    assert np.array_equal(a[0], b[0]) and not np.array_equal(a[0], c[0])


def test_frequency_weights():
    # hist(v)^-alpha over the values present, mean 1, absent values 0: over
    # the images' own pixels, alpha = 1 gives every present value the same
    # total weight, alpha = 0 weight 1 per pixel (the plain loss)
    from paper_2207_05152_gb300 import train as T
    imgs = [synth.phantom_image(48, 40, 60 + i) for i in range(2)]
    flat = np.concatenate([im.reshape(-1) for im in imgs])
    hist = np.bincount(flat, minlength=256)
    w = T.frequency_weights(imgs, 1.0).astype(np.float64)
    present = hist > 0
    assert np.all(w[~present] == 0) and np.all(w[present] > 0)
    assert abs(w[present].mean() - 1.0) < 1e-6
    totals = (hist * w)[present]
    assert np.allclose(totals, totals[0], rtol=1e-5)
    w0 = T.frequency_weights(imgs, 0.0)
    assert np.all(w0[present] == 1.0) and np.all(w0[~present] == 0)
