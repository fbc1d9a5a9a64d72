"""Pins of the oracle's PDF -> frequency-table quantisation.

The coder needs an integer table per pixel that sums to 2^16 with every entry
at least 1 (so every 8-bit value stays codable) and that follows the
network's softmax PDF (Sec. II-B: 256 softmax outputs, one per grey value).
These tests check the oracle's table against closed forms and against an
independent float64 softmax."""
import numpy as np
import pytest

import synth
from paper_2207_05152_gb300 import model as M

TS = float(M.TSCALE)
LUT = M.table_lut()


def _freqs(orc, z):
    cum = orc.table_from_logits(np.asarray(z, np.float32), TS, LUT)
    return cum, np.diff(cum.astype(np.int64))


def test_lut_matches_its_formula():
    k = np.arange(64)
    exact = 2.0 ** (23 - k / 64)
    assert LUT[0] == 1 << 23
    assert np.all(np.abs(LUT - exact) <= 0.5)
    assert np.all(np.diff(LUT.astype(np.int64)) < 0)


@pytest.mark.parametrize("spread", [0.0, 0.01, 0.5, 2.0, 8.0, 40.0, 1e4])
def test_table_invariants(orc, spread):
    rng = synth.Rng(int(spread * 100) + 3)
    for _ in range(50):
        z = rng.normal(256) * spread
        cum, f = _freqs(orc, z)
        assert cum[0] == 0 and cum[256] == 65536
        assert f.sum() == 65536
        assert f.min() >= 1
        assert f.max() <= 65281


def test_uniform_logits_give_flat_table(orc):
    # All logits equal: every weight is lut[0] = 2^23, W = 2^31, Q = 130560,
    # c_i = i + 255 i = 256 i, so f_i = 256 exactly (8 bits per symbol).
    for v in (0.0, -3.5, 1e6):
        cum, f = _freqs(orc, np.full(256, v))
        assert np.all(f == 256)
        assert np.array_equal(cum, 256 * np.arange(257))


@pytest.mark.parametrize("k", [0, 1, 77, 254, 255])
def test_dominant_logit(orc, k):
    # One logit far above the rest: every other weight underflows to 0, so
    # the dominant symbol gets 2^16 - 255 and every other symbol exactly 1.
    z = np.zeros(256)
    z[k] = 1000.0
    _, f = _freqs(orc, z)
    assert f[k] == 65281
    assert np.all(np.delete(f, k) == 1)


def test_tied_maxima_share_mass(orc):
    z = np.full(256, -1000.0)
    z[[3, 200]] = 5.0
    _, f = _freqs(orc, z)
    assert abs(int(f[3]) - int(f[200])) <= 1
    assert f[3] + f[200] == 65536 - 254


@pytest.mark.parametrize("spread", [0.3, 1.0, 3.0, 10.0])
def test_table_follows_softmax(orc, spread):
    # |f_i / 2^16 - p_i| <= 0.015 p_i + 3 / 2^16: the log2 grid of 1/64
    # (factor 2^(+-1/128)) on each weight, the floor of the cumulative
    # quantisation (+-1) and the "+1" floor of every entry.
    rng = synth.Rng(99 + int(spread * 10))
    for _ in range(40):
        z = (rng.normal(256) * spread).astype(np.float32)
        _, f = _freqs(orc, z)
        zz = z.astype(np.float64)
        p = np.exp(zz - zz.max())
        p /= p.sum()
        err = np.abs(f / 65536.0 - p)
        assert np.all(err <= 0.015 * p + 3.0 / 65536.0), err.max()


def test_table_is_monotone_in_logits(orc):
    rng = synth.Rng(5)
    z = rng.normal(256) * 4
    _, f = _freqs(orc, z)
    order = np.argsort(z, kind="stable")
    # A larger logit never gets a frequency smaller by more than the one
    # count of cumulative rounding.
    fs = f[order].astype(np.int64)
    assert np.all(np.diff(fs) >= -1)
