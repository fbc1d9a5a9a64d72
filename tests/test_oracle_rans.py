"""Pins of the oracle's rANS coder (Sec. II-B "rANS").

The coder step must be a bijection between (state, symbol) and (new state,
renormalisation words), so that the decoder undoes the encoder exactly.  At
reduced bit widths every state can be enumerated; at the coder's own widths
(32-bit state, 16-bit words, tables of 2^16) random and boundary states are
checked, together with the single-word renormalisation property that 32-bit
arithmetic relies on."""
import numpy as np
import pytest

import synth


def _random_cum(rng, nsym, total):
    f = np.ones(nsym, np.int64)
    extra = total - nsym
    cuts = np.sort(rng.integers(nsym - 1, 0, extra))
    f += np.diff(np.concatenate([[0], cuts, [extra]]))
    return np.concatenate([[0], np.cumsum(f)]).astype(np.uint32)


@pytest.mark.parametrize("Lb,bb,Mb,nsym", [(8, 4, 4, 16), (6, 2, 4, 5), (7, 6, 6, 3), (9, 3, 6, 20)])
def test_step_is_a_bijection_exhaustive(orc, Lb, bb, Mb, nsym):
    rng = synth.Rng(Lb * 100 + bb * 10 + Mb)
    cum = _random_cum(rng, nsym, 1 << Mb)
    L, b = 1 << Lb, 1 << bb
    seen = {}
    for x in range(L, L * b):
        for s in range(nsym):
            f, c = int(cum[s + 1] - cum[s]), int(cum[s])
            y, words = orc.rans_enc_step(x, f, c, Lb, bb, Mb)
            assert L <= y < L * b
            key = (y, tuple(words))
            assert key not in seen
            seen[key] = (x, s)
            # decoder reads the words in reverse emission order
            s2, x2, pos = orc.rans_dec_step(y, cum, list(reversed(words)), 0, Lb, bb, Mb)
            assert (s2, x2, pos) == (s, x, len(words))
    # every (state, words) pair the decoder can meet comes from exactly one
    # encoder step: decode then encode gives back the same state and words
    for y in range(L, L * b):
        for w in range(min(b, 8)):
            words = [w, (w * 7 + 3) % b, (w * 5 + 1) % b]
            s, x, pos = orc.rans_dec_step(y, cum, words, 0, Lb, bb, Mb)
            assert 0 <= s < nsym and L <= x < L * b
            f, c = int(cum[s + 1] - cum[s]), int(cum[s])
            y2, em = orc.rans_enc_step(x, f, c, Lb, bb, Mb)
            assert y2 == y and em[::-1] == words[:pos]


def test_coder_widths_single_word_renorm(orc):
    rng = synth.Rng(17)
    cum = _random_cum(rng, 256, 1 << 16)
    states = list(rng.integers(2000, 1 << 16, (1 << 32) - 1)) + [1 << 16, (1 << 32) - 1, (1 << 24)]
    for x in states:
        for s in (0, 1, 127, 255):
            f, c = int(cum[s + 1] - cum[s]), int(cum[s])
            y, words = orc.rans_enc_step(int(x), f, c)
            assert len(words) <= 1
            assert (1 << 16) <= y < (1 << 32)
            s2, x2, _ = orc.rans_dec_step(y, cum, words[::-1], 0)
            assert (s2, x2) == (s, int(x))
    # extreme frequencies: f = 1 and f = 2^16 - 255
    for f, c in ((1, 0), (65281, 255)):
        for x in ((1 << 16), (1 << 32) - 1, (f << 16) - 1, f << 16):
            if x >= 1 << 32:
                continue
            y, words = orc.rans_enc_step(x, f, c)
            assert len(words) <= 1 and y < (1 << 32)


def test_sequence_roundtrip_and_length(orc):
    # Encode a sequence in reverse, decode forward; the output length in bits
    # tracks the ideal code length sum -log2(f/M).
    rng = synth.Rng(23)
    cum = _random_cum(rng, 256, 1 << 16)
    f = np.diff(cum.astype(np.int64))
    p = f / 65536.0
    syms = rng.integers(20000, 0, 255)
    x, emitted = 1 << 16, []
    for s in syms[::-1]:
        x, w = orc.rans_enc_step(x, int(f[s]), int(cum[s]))
        emitted += w
    words = emitted[::-1]
    out, pos, y = [], 0, x
    for _ in syms:
        s, y, pos = orc.rans_dec_step(y, cum, words, pos)
        out.append(s)
    assert out == list(syms) and y == 1 << 16 and pos == len(words)
    bits = 16 * len(words) + np.log2(x) - 16
    ideal = -np.log2(p[syms]).sum()
    assert abs(bits - ideal) / len(syms) < 0.01
