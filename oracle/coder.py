"""ctypes wrapper of the C oracle (dlic_oracle.c).  Test infrastructure only:
the functions here restate the coding method sequentially on the CPU and are
what the CUDA library is checked against."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dlic_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

U8P = C.POINTER(C.c_uint8)
U16P = C.POINTER(C.c_uint16)
VP = C.c_void_p
U32P = C.POINTER(C.c_uint32)
F32P = C.POINTER(C.c_float)
F64P = C.POINTER(C.c_double)
U64P = C.POINTER(C.c_uint64)
IP = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (IEEE, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_fnv1a64.restype = C.c_uint64
            L.or_fnv1a64.argtypes = [U8P, C.c_size_t]
            L.or_gather.restype = None
            L.or_gather.argtypes = [U8P, C.c_int, C.c_int, C.c_int, C.c_int, U8P]
            L.or_gather_window.restype = C.c_int
            L.or_gather_window.argtypes = [C.c_int, C.c_int, C.c_int, U8P, C.c_int, C.c_int, C.c_int, C.c_int, U8P]
            L.or_table_from_logits.restype = C.c_int
            L.or_table_from_logits.argtypes = [F32P, C.c_float, U32P, U32P]
            L.or_table_k.restype = C.c_int
            L.or_table_k.argtypes = [F32P, C.c_int, C.c_float, U32P, U32P]
            L.or_rans_enc_step.restype = C.c_int
            L.or_rans_enc_step.argtypes = [U64P, C.c_uint32, C.c_uint32, C.c_int, C.c_int, C.c_int,
                                           U32P, C.c_int]
            L.or_rans_dec_step.restype = C.c_int
            L.or_rans_dec_step.argtypes = [U64P, U32P, C.c_int, C.c_int, C.c_int, C.c_int, U32P,
                                           C.c_int, IP]
            L.or_max_encoded_bytes.restype = C.c_size_t
            L.or_max_encoded_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
            L.or_pixel_table.restype = C.c_int
            L.or_pixel_table.argtypes = [U8P, C.c_size_t, VP, C.c_int, C.c_int, C.c_int, C.c_int,
                                         F32P, U32P]
            L.or_logits.restype = C.c_int
            L.or_logits.argtypes = [U8P, C.c_size_t, U16P, C.c_int, F32P]
            L.or_symbol_tables.restype = C.c_int
            L.or_symbol_tables.argtypes = [U8P, C.c_size_t, VP, C.c_int, C.c_int, U32P, F64P]
            L.or_encode.restype = C.c_int64
            L.or_encode.argtypes = [U8P, C.c_size_t, VP, C.c_int, C.c_int, C.c_int, U8P,
                                    C.c_size_t]
            L.or_decode.restype = C.c_int
            L.or_decode.argtypes = [U8P, C.c_size_t, U8P, C.c_size_t, VP, C.c_int, C.c_int]
            L.or_gather_window3.restype = C.c_int
            L.or_gather_window3.argtypes = [C.c_int] * 7 + [U8P, U8P, C.c_int, C.c_int, C.c_int, C.c_int, U8P]
            L.or_encode_volume.restype = C.c_int64
            L.or_encode_volume.argtypes = [U8P, C.c_size_t, VP, C.c_int, C.c_int, C.c_int, C.c_int, U8P,
                                           C.c_size_t, U64P]
            L.or_decode_volume.restype = C.c_int
            L.or_decode_volume.argtypes = [U8P, C.c_size_t, U8P, U64P, C.c_int, VP, C.c_int, C.c_int]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _bytes(b) -> np.ndarray:
    return np.frombuffer(bytes(b), dtype=np.uint8).copy()


def symbols(blob: bytes) -> int:
    """Output neurons of a model blob: 256 (8-bit pixels) or 4096 (12-bit)."""
    off = 48 if bytes(blob[:4]) == b"DLM2" else 20
    return int(np.frombuffer(bytes(blob[off:off + 4]), "<u4")[0])


def _pixels(blob: bytes, img) -> np.ndarray:
    """img as the model's sample type: u8 for 8-bit, u16 for 12-bit pixels."""
    return np.ascontiguousarray(img, dtype=np.uint16 if symbols(blob) == 4096 else np.uint8)


def fnv1a64(data: bytes) -> int:
    a = _bytes(data)
    return int(lib().or_fnv1a64(_p(a, U8P), a.size))


def max_encoded_bytes(H: int, W: int, S: int) -> int:
    return int(lib().or_max_encoded_bytes(H, W, S))


def gather(img: np.ndarray, r: int, c: int) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    out = np.zeros(12, np.uint8)
    lib().or_gather(_p(img, U8P), img.shape[0], img.shape[1], r, c, _p(out, U8P))
    return out


def gather_window(window, img: np.ndarray, r: int, c: int) -> np.ndarray:
    """Priors of pixel (r, c) for the causal window (u, l, r_reach)."""
    u, l, rr = window
    img = np.ascontiguousarray(img, dtype=np.uint8)
    out = np.zeros(u * (l + rr + 1) + l, np.uint8)
    n = lib().or_gather_window(u, l, rr, _p(img, U8P), img.shape[0], img.shape[1], r, c, _p(out, U8P))
    assert n == out.size
    return out


def gather_window3(window, below, img: np.ndarray, r: int, c: int) -> np.ndarray:
    """Priors of pixel (r, c) of a slice for the 3D window (u, l, r_reach,
    pu, pd, pl, pr); below is the previous slice, or None for the first."""
    u, l, rr, pu, pd, pl, pr = window
    img = np.ascontiguousarray(img, dtype=np.uint8)
    n = u * (l + rr + 1) + l + (pu + pd + 1) * (pl + pr + 1)
    out = np.zeros(n, np.uint8)
    bp = _p(np.ascontiguousarray(below, dtype=np.uint8), U8P) if below is not None else None
    got = lib().or_gather_window3(u, l, rr, pu, pd, pl, pr, bp, _p(img, U8P), img.shape[0], img.shape[1], r, c,
                                  _p(out, U8P))
    assert got == n
    return out


def table_from_logits(z, tscale: float, lut) -> np.ndarray:
    """Cumulative table c_0..c_K (uint32) for one logit vector of K symbols
    (256, or 4096 for 12-bit pixels)."""
    z = np.ascontiguousarray(z, dtype=np.float32).reshape(-1)
    lut = np.ascontiguousarray(lut, dtype=np.uint32)
    cum = np.zeros(z.size + 1, np.uint32)
    st = lib().or_table_k(_p(z, F32P), z.size, C.c_float(tscale), _p(lut, U32P), _p(cum, U32P))
    if st:
        raise ValueError(f"oracle table error {st}")
    return cum


def rans_enc_step(x: int, f: int, c: int, Lb=16, bb=16, Mb=16):
    xs = (C.c_uint64 * 1)(x)
    em = (C.c_uint32 * 8)()
    n = lib().or_rans_enc_step(xs, f, c, Lb, bb, Mb, em, 8)
    if n < 0:
        raise ValueError("too many renormalisation words")
    return int(xs[0]), [int(em[i]) for i in range(n)]


def rans_dec_step(x: int, cum, words, pos: int, Lb=16, bb=16, Mb=16):
    cum = np.ascontiguousarray(cum, dtype=np.uint32)
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).reshape(-1))
    if w.size == 0:
        w = np.zeros(1, np.uint32)
        nw = 0
    else:
        nw = w.size
    xs = (C.c_uint64 * 1)(x)
    ps = (C.c_int * 1)(pos)
    s = lib().or_rans_dec_step(xs, _p(cum, U32P), cum.size - 1, Lb, bb, Mb, _p(w, U32P), nw, ps)
    return s, int(xs[0]), int(ps[0])


def pixel_table(blob: bytes, img: np.ndarray, r: int, c: int):
    """(logits[K] float32, cum[K + 1] uint32) of pixel (r, c), K the model's
    symbol count."""
    b = _bytes(blob)
    img = _pixels(blob, img)
    K = symbols(blob)
    z = np.zeros(K, np.float32)
    cum = np.zeros(K + 1, np.uint32)
    st = lib().or_pixel_table(_p(b, U8P), b.size, img.ctypes.data, img.shape[0], img.shape[1], r, c,
                              _p(z, F32P), _p(cum, U32P))
    if st:
        raise ValueError(f"oracle error {st}")
    return z, cum


def logits(blob: bytes, pri: np.ndarray) -> np.ndarray:
    """Logits [n, K] for prior vectors [n, window size] (sample values)."""
    b = _bytes(blob)
    n_in = int(np.frombuffer(b[8:12].tobytes(), "<u4")[0])
    pri = np.ascontiguousarray(pri, dtype=np.uint16).reshape(-1, n_in)
    z = np.zeros((pri.shape[0], symbols(blob)), np.float32)
    st = lib().or_logits(_p(b, U8P), b.size, _p(pri, U16P), pri.shape[0], _p(z, F32P))
    if st:
        raise ValueError(f"oracle error {st}")
    return z


def symbol_tables(blob: bytes, img: np.ndarray):
    """(f | c << 16 per pixel as uint32 [H, W], ideal bits sum -log2(f/2^16))."""
    b = _bytes(blob)
    img = _pixels(blob, img)
    fc = np.zeros(img.shape, np.uint32)
    bits = (C.c_double * 1)()
    st = lib().or_symbol_tables(_p(b, U8P), b.size, img.ctypes.data, img.shape[0], img.shape[1],
                                _p(fc, U32P), bits)
    if st:
        raise ValueError(f"oracle error {st}")
    return fc, float(bits[0])


def encode(blob: bytes, img: np.ndarray, streams: int) -> bytes:
    """The container of one image (u8 samples, or u16 for a 12-bit model)."""
    b = _bytes(blob)
    img = _pixels(blob, img)
    H, W = img.shape
    cap = max_encoded_bytes(H, W, streams)
    out = np.zeros(cap, np.uint8)
    n = lib().or_encode(_p(b, U8P), b.size, img.ctypes.data, H, W, streams, _p(out, U8P), cap)
    if n < 0:
        raise ValueError(f"oracle encode error {-n}")
    return out[:n].tobytes()


def decode(blob: bytes, data: bytes, H: int, W: int):
    """(status, image): status 0 on success, 3 for a corrupt stream."""
    b = _bytes(blob)
    d = _bytes(data)
    if d.size == 0:
        d = np.zeros(1, np.uint8)
        n = 0
    else:
        n = d.size
    img = np.zeros((H, W), np.uint16 if symbols(blob) == 4096 else np.uint8)
    st = lib().or_decode(_p(b, U8P), b.size, _p(d, U8P), n, img.ctypes.data, H, W)
    return int(st), img


def encode_volume(blob: bytes, vol: np.ndarray, streams: int):
    """(bytes, offsets): the D slice containers of a volume (D x H x W)
    coded with a 3D window, back to back, and the D + 1 byte offsets."""
    b = _bytes(blob)
    vol = _pixels(blob, vol)
    D, H, W = vol.shape
    cap = D * max_encoded_bytes(H, W, streams)
    out = np.zeros(cap, np.uint8)
    offs = np.zeros(D + 1, np.uint64)
    n = lib().or_encode_volume(_p(b, U8P), b.size, vol.ctypes.data, D, H, W, streams, _p(out, U8P), cap,
                               _p(offs, U64P))
    if n < 0:
        raise ValueError(f"oracle encode error {-n}")
    return out[:n].tobytes(), [int(o) for o in offs]


def decode_volume(blob: bytes, data: bytes, offsets, D: int, H: int, W: int):
    """(status, volume D x H x W) of a volume coded by encode_volume."""
    b = _bytes(blob)
    d = _bytes(data) if len(data) else np.zeros(1, np.uint8)
    offs = np.asarray(offsets, dtype=np.uint64)
    vol = np.zeros((D, H, W), np.uint16 if symbols(blob) == 4096 else np.uint8)
    st = lib().or_decode_volume(_p(b, U8P), b.size, _p(d, U8P), _p(offs, U64P), D, vol.ctypes.data, H, W)
    return int(st), vol
