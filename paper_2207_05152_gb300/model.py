"""Model blobs for the DLIC coder: serialisation and post-training quantisation.

The density-estimation network (Sec. II-B, "Neural Network Architecture") maps
the 12 causal priors of a pixel to 256 logits, one per 8-bit value; the
softmax of those logits is the PDF the entropy coder uses (Eq. 1).  The coder
needs that PDF to be bit-identical at encode and decode (Sec. II-B,
"Preprocessor": the same matrices must enter the network on both sides), so a
model is shipped as one little-endian byte blob that fixes every number the
coder uses:

    0    char[4] "DLM1"
    4    u32 precision            0 = FP32 network, 1 = INT8 network
    8    u32 n_in, n_h1, n_h2, n_out, window
         n_out = 256 for 8-bit pixels, 4096 for 12-bit pixels (Sec. IV
         "Higher Bit Depth"; FP32 networks only, input v / 2048 - 1)
         window = 2: the default radius-2 window (n_in = 12); otherwise
         1 << 24 | u | l << 8 | r << 16: rows r-u..r-1 at columns c-l..c+r,
         then row r at columns c-l..c-1 (n_in = u (l + r + 1) + l, at most
         96; u <= 8, l <= 8, r <= 2); or a 3D window (Sec. IV "3D
         Dependencies") 2 << 28 | u | l << 4 | r << 8 | pu << 10 | pd << 14 |
         pl << 18 | pr << 22: the 2D window, then from the previous slice
         rows r-pu..r+pd at columns c-pl..c+pr (pu, pd, pl, pr <= 8)
    28   f32 tscale               logit difference -> table units (64 / ln 2)
    32   u32 lut[64]              lut[k] = round(2^23 * 2^(-k/64)), lut[0] = 2^23
    288  layer data
         FP32: W1 f32[h1][n_in], b1 f32[h1], W2 f32[h2][h1], b2 f32[h2],
               W3 f32[256][h2], b3 f32[256]
         INT8: W1 i8[h1][n_in], s1 f32[h1], o1 f32[h1],
               W2 i8[h2][h1], s2 f32[h2], o2 f32[h2],
               W3 i8[256][h2], s3 f32[256], o3 f32[256]

The INT8 network computes, per layer, an exact integer dot product
acc = sum_k Wq[j][k] * a_k (inputs are v - 128 for the priors and u8 hidden
activations), then h_j = clamp(rint(fma(acc, s_j, o_j)), 0, 255) for hidden
layers and z_j = fma(acc, s_j, o_j) for the logits.  This module holds the
host-side model preparation only; every coding step runs in the CUDA library.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"DLM1"
PREC_FP32 = 0
PREC_INT8 = 1
N_IN = 12
N_OUT = 256
N_OUT_12 = 4096   # 12-bit pixels: one output neuron per value (Sec. IV "Higher Bit Depth")
RADIUS = 2
DEFAULT_WINDOW = (2, 2, 2)
FIG6_WINDOW = (8, 6, 2)   # 9 x 9 window, target in the last row, third column from the right
# 3D window: the default 2D window plus the 3 x 3 neighbourhood of the pixel
# in the previous slice (one row below the target's row: the lower layer is
# shifted down, Sec. IV "3D Wavefront")
VOLUME_WINDOW = (2, 2, 2, 1, 1, 1, 1)


def is_volume(window) -> bool:
    return len(window) == 7


def window_size(window) -> int:
    u, l, r = window[:3]
    n = u * (l + r + 1) + l
    if is_volume(window):
        pu, pd, pl, pr = window[3:]
        n += (pu + pd + 1) * (pl + pr + 1)
    return n


def volume_wave_shift(window) -> int:
    """Waves by which slice z + 1 lags slice z in the 3D wavefront: the
    smallest shift that puts every prior of the previous slice on an earlier
    wave, 3 pd + pr + 1 (the lower layer's reach below and right)."""
    pd, pr = window[4], window[6]
    return 3 * pd + pr + 1


def window_offsets(window) -> list:
    """(row, column) offset of every prior of the causal window (u rows
    above, l columns left, r right; Sec. II-A), in the network's input
    order: the rows above top to bottom, each left to right, then the l
    pixels left of the target."""
    u, l, r = window[:3]
    span = l + r + 1
    return [(k // span - u, k % span - l) for k in range(u * span)] + [(0, k - l) for k in range(l)]


def window_offsets3(window) -> list:
    """(slice, row, column) offset of every prior of a 2D or 3D window, in
    the network's input order: the 2D window in the pixel's own slice
    (slice offset 0), then for a 3D window the previous slice's rows
    r-pu..r+pd, each at columns c-pl..c+pr (slice offset -1)."""
    offs = [(0, dr, dc) for dr, dc in window_offsets(window[:3])]
    if is_volume(window):
        pu, pd, pl, pr = window[3:]
        offs += [(-1, dr, dc) for dr in range(-pu, pd + 1) for dc in range(-pl, pr + 1)]
    return offs


def window_field(window) -> int:
    """The blob's window field: 2 for the default window, else the packed
    (u, l, r)."""
    window = tuple(int(v) for v in window)
    if is_volume(window):
        u, l, r, pu, pd, pl, pr = window
        if not (1 <= u <= 8 and 0 <= l <= 8 and 0 <= r <= 2 and max(pu, pd, pl, pr) <= 8 and min(window) >= 0) \
                or window_size(window) > 96:
            raise ValueError("3D window must have 1 <= u <= 8, l <= 8, r <= 2, pu, pd, pl, pr <= 8 and at most "
                             "96 priors")
        return (2 << 28) | u | (l << 4) | (r << 8) | (pu << 10) | (pd << 14) | (pl << 18) | (pr << 22)
    if window == DEFAULT_WINDOW:
        return RADIUS
    u, l, r = window
    if not (1 <= u <= 8 and 0 <= l <= 8 and 0 <= r <= 2) or window_size(window) > 96:
        raise ValueError("window must have 1 <= u <= 8, l <= 8, r <= 2 and at most 96 priors")
    return (1 << 24) | u | (l << 8) | (r << 16)


def window_of_field(field: int):
    if field == RADIUS:
        return DEFAULT_WINDOW
    if field >> 28 == 2:
        return (field & 0xF, (field >> 4) & 0xF, (field >> 8) & 3, (field >> 10) & 0xF, (field >> 14) & 0xF,
                (field >> 18) & 0xF, (field >> 22) & 0xF)
    if field >> 24 != 1:
        raise ValueError("unknown window field")
    return (field & 0xFF, (field >> 8) & 0xFF, (field >> 16) & 0xFF)
HEADER_BYTES = 288
TSCALE = np.float32(64.0 / np.log(2.0))


def table_lut() -> np.ndarray:
    """lut[k] = round(2^23 * 2^(-k/64)), k = 0..63: the fixed-point powers of
    two the table quantisation uses to turn log2-domain logit gaps into
    relative weights."""
    k = np.arange(64, dtype=np.float64)
    return np.rint(np.exp2(23.0 - k / 64.0)).astype(np.uint32)


def _header(precision: int, h1: int, h2: int, window=DEFAULT_WINDOW, n_out: int = N_OUT) -> bytes:
    hdr = MAGIC + struct.pack("<6I", precision, window_size(window), h1, h2, n_out, window_field(window))
    hdr += struct.pack("<f", float(TSCALE))
    hdr += table_lut().astype("<u4").tobytes()
    assert len(hdr) == HEADER_BYTES
    return hdr


def _check_widths(layers, window=DEFAULT_WINDOW, n_out: int = N_OUT):
    if len(layers) != 3:
        raise ValueError("the coder network has exactly three dense layers")
    (w1, b1), (w2, b2), (w3, b3) = layers
    h1, h2 = w1.shape[0], w2.shape[0]
    if w1.shape != (h1, window_size(window)) or w2.shape != (h2, h1) or w3.shape != (n_out, h2):
        raise ValueError(f"layer shapes must be (h1, window size), (h2, h1), ({n_out}, h2)")
    if b1.shape != (h1,) or b2.shape != (h2,) or b3.shape != (n_out,):
        raise ValueError("bias shapes do not match the layers")
    if h1 % 16 or h2 % 16 or not (16 <= h1 <= 256) or not (16 <= h2 <= 256):
        raise ValueError("hidden widths must be multiples of 16 in [16, 256]")
    return h1, h2


def fp32_blob(layers, window=DEFAULT_WINDOW) -> bytes:
    """Blob of an FP32 network given [(W1, b1), (W2, b2), (W3, b3)] for the
    causal window (u, l, r)."""
    h1, h2 = _check_widths(layers, window)
    out = [_header(PREC_FP32, h1, h2, window)]
    for w, b in layers:
        out.append(np.ascontiguousarray(w, dtype="<f4").tobytes())
        out.append(np.ascontiguousarray(b, dtype="<f4").tobytes())
    return b"".join(out)


def model_symbols(blob: bytes) -> int:
    """Output neurons of a "DLM1" or "DLM2" blob: 256 (8-bit pixels) or 4096."""
    off = 48 if bytes(blob[:4]) == DEEP_MAGIC else 20
    return struct.unpack_from("<I", blob, off)[0]


def fp32_blob12(layers) -> bytes:
    """Blob of an FP32 network for 12-bit pixels, [(W1, b1), (W2, b2),
    (W3, b3)] with 4096 outputs, over the default window."""
    h1, h2 = _check_widths(layers, DEFAULT_WINDOW, N_OUT_12)
    out = [_header(PREC_FP32, h1, h2, DEFAULT_WINDOW, N_OUT_12)]
    for w, b in layers:
        out.append(np.ascontiguousarray(w, dtype="<f4").tobytes())
        out.append(np.ascontiguousarray(b, dtype="<f4").tobytes())
    return b"".join(out)


def features_fp32(ctx_u8: np.ndarray) -> np.ndarray:
    """Network input for 8-bit priors: v / 128 - 1."""
    return ctx_u8.astype(np.float32) / np.float32(128.0) - np.float32(1.0)


def _forward_fp32(layers, ctx_u8):
    x = features_fp32(ctx_u8).astype(np.float64)
    acts = []
    for li, (w, b) in enumerate(layers):
        x = x @ w.astype(np.float64).T + b.astype(np.float64)
        if li < len(layers) - 1:
            x = np.maximum(x, 0.0)
            acts.append(x)
    return acts, x


def _quantise(layers, calib_ctx):
    """Per-layer (Wq, s, o) of the post-training quantisation (any depth)."""
    acts, _ = _forward_fp32(layers, np.asarray(calib_ctx, dtype=np.uint8))
    act_scale = [max(float(a.max()), 1e-6) / 255.0 for a in acts]
    in_scale = [1.0 / 128.0] + act_scale
    out = []
    for li, (w, b) in enumerate(layers):
        w = w.astype(np.float64)
        b = b.astype(np.float64)
        sw = np.abs(w).max(axis=1) / 127.0
        sw[sw == 0] = 1.0
        wq = np.clip(np.rint(w / sw[:, None]), -127, 127).astype(np.int8)
        if li < len(layers) - 1:
            s = sw * in_scale[li] / act_scale[li]
            o = b / act_scale[li]
        else:
            s = sw * in_scale[li]
            o = b
        out.append((wq, s, o))
    return out


def int8_blob(layers, calib_ctx: np.ndarray, window=DEFAULT_WINDOW) -> bytes:
    """Post-training quantisation of an FP32 network to the INT8 blob.

    Weights: per-output-channel symmetric scale max|w| / 127, round half to
    even, clamp to +-127.  Hidden activations: u8 with a per-layer scale
    max(h) / 255 over the calibration contexts (u8 array [N, window size]).
    Inputs: v - 128 with scale 1/128."""
    h1, h2 = _check_widths(layers, window)
    out = [_header(PREC_INT8, h1, h2, window)]
    for wq, s, o in _quantise(layers, calib_ctx):
        out.append(wq.tobytes())
        out.append(s.astype("<f4").tobytes())
        out.append(o.astype("<f4").tobytes())
    return b"".join(out)


# --- deeper networks (Sec. II-B "Neural Network Architecture": six dense
# layers): the "DLM2" blob, L hidden layers of any widths up to 4096 ---
DEEP_MAGIC = b"DLM2"
DEEP_HEADER_BYTES = 320
MAX_HIDDEN_LAYERS = 8


def _deep_header(precision: int, widths, window, n_out: int = N_OUT) -> bytes:
    L = len(widths)
    hdr = DEEP_MAGIC + struct.pack("<3I", precision, window_size(window), L)
    hdr += struct.pack("<8I", *(list(widths) + [0] * (MAX_HIDDEN_LAYERS - L)))
    hdr += struct.pack("<2IfI", n_out, window_field(window), float(TSCALE), 0)
    hdr += table_lut().astype("<u4").tobytes()
    assert len(hdr) == DEEP_HEADER_BYTES
    return hdr


def _check_deep(layers, window):
    if not 2 <= len(layers) <= MAX_HIDDEN_LAYERS + 1:
        raise ValueError("a deep network has 1 to 8 hidden layers and the output layer")
    widths, n = [], window_size(window)
    for li, (w, b) in enumerate(layers):
        if w.ndim != 2 or w.shape[1] != n or b.shape != (w.shape[0],):
            raise ValueError(f"layer {li}: shape {w.shape} does not chain from {n} inputs")
        n = w.shape[0]
        if li < len(layers) - 1:
            if not 1 <= n <= 4096:
                raise ValueError("hidden widths must be in [1, 4096]")
            widths.append(n)
    if n not in (N_OUT, N_OUT_12):
        raise ValueError("the output layer has 256 units (4096 for 12-bit pixels)")
    return widths


def deep_fp32_blob(layers, window=DEFAULT_WINDOW) -> bytes:
    """"DLM2" blob of an FP32 network [(W1, b1), ..., (W_out, b_out)] of
    1..8 hidden layers (256 outputs, or 4096 for 12-bit pixels)."""
    out = [_deep_header(PREC_FP32, _check_deep(layers, window), window, layers[-1][0].shape[0])]
    for w, b in layers:
        out.append(np.ascontiguousarray(w, dtype="<f4").tobytes())
        out.append(np.ascontiguousarray(b, dtype="<f4").tobytes())
    return b"".join(out)


def deep_int8_blob(layers, calib_ctx: np.ndarray, window=DEFAULT_WINDOW) -> bytes:
    """"DLM2" blob of the INT8 quantisation (the rules of int8_blob) of a
    network of 1..8 hidden layers."""
    if layers[-1][0].shape[0] != N_OUT:
        raise ValueError("an INT8 network has 256 outputs (8-bit pixels)")
    out = [_deep_header(PREC_INT8, _check_deep(layers, window), window)]
    for wq, s, o in _quantise(layers, calib_ctx):
        out.append(wq.tobytes())
        out.append(s.astype("<f4").tobytes())
        out.append(o.astype("<f4").tobytes())
    return b"".join(out)


def parse_blob(blob: bytes) -> dict:
    """Split a blob into its named arrays (for inspection and training)."""
    if blob[:4] != MAGIC:
        raise ValueError("not a DLIC model blob")
    prec, n_in, h1, h2, n_out, radius = struct.unpack_from("<6I", blob, 4)
    (tscale,) = struct.unpack_from("<f", blob, 28)
    lut = np.frombuffer(blob, dtype="<u4", count=64, offset=32)
    d = dict(precision=prec, n_in=n_in, h1=h1, h2=h2, n_out=n_out, radius=radius,
             window=window_of_field(radius), tscale=tscale, lut=lut)
    off = HEADER_BYTES
    dims = [(h1, n_in), (h2, h1), (n_out, h2)]
    for li, (o, i) in enumerate(dims, start=1):
        if prec == PREC_FP32:
            d[f"W{li}"] = np.frombuffer(blob, "<f4", o * i, off).reshape(o, i); off += 4 * o * i
            d[f"b{li}"] = np.frombuffer(blob, "<f4", o, off); off += 4 * o
        else:
            d[f"Q{li}"] = np.frombuffer(blob, "i1", o * i, off).reshape(o, i); off += o * i
            d[f"s{li}"] = np.frombuffer(blob, "<f4", o, off); off += 4 * o
            d[f"o{li}"] = np.frombuffer(blob, "<f4", o, off); off += 4 * o
    if off != len(blob):
        raise ValueError("blob size does not match its header")
    return d

