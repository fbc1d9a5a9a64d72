"""ctypes binding of libdlic.so: the C-ABI entry points under the same names.

Argument marshalling only; every step of the coding path runs in the CUDA
library.  Loading fails loudly when the library has not been built."""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdlic.so")
_lock = threading.Lock()
_lib = None

DLIC_OK, DLIC_ERR_INVALID, DLIC_ERR_CAPACITY, DLIC_ERR_CORRUPT = 0, 1, 2, 3
DLIC_ERR_TIMEOUT, DLIC_ERR_CUDA, DLIC_ERR_UNSUPPORTED = 4, 5, 6
DLIC_FP32, DLIC_INT8 = 0, 1
DLIC_TRAIN_BF16, DLIC_TRAIN_FP32, DLIC_TRAIN_BF16X3 = 0, 1, 2
DLIC_TRAIN_RECOMPUTE = 0x100
DLIC_PLAN_AUTO, DLIC_PLAN_BYTE_RING, DLIC_PLAN_IMAGE, DLIC_PLAN_GRID = 0, 1, 2, 3


class DlicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dlic error {code}: {msg}")
        self.code = code


class dlic_image(C.Structure):
    _fields_ = [("pixels", C.c_void_p), ("height", C.c_int32), ("width", C.c_int32),
                ("pitch", C.c_int64)]


class dlic_volume(C.Structure):
    _fields_ = [("pixels", C.c_void_p), ("depth", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("streams", C.c_int32), ("pitch", C.c_int64), ("slice_pitch", C.c_int64)]


_VP = C.c_void_p
_SZ = C.c_size_t
_I = C.c_int
_VOLP = C.POINTER(dlic_volume)
_IMGP = C.POINTER(dlic_image)

# name -> (restype, argtypes); every symbol include/dlic.h declares
SIGNATURES = {
    "dlic_last_error": (C.c_char_p, []),
    "dlic_model_create": (_I, [_VP, _SZ, C.POINTER(_VP)]),
    "dlic_model_destroy": (_I, [_VP]),
    "dlic_model_set_decode_plan": (_I, [_VP, _I]),
    "dlic_model_set_peer_wait_limit": (_I, [_VP, C.c_longlong]),
    "dlic_model_info": (_I, [_VP, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(C.c_uint64)]),
    "dlic_max_encoded_bytes": (_SZ, [_I, _I, _I]),
    "dlic_auto_streams": (_I, [_I, _I]),
    "dlic_encode_workspace_size": (_I, [_VP, _IMGP, _I, C.POINTER(_I), C.POINTER(_SZ)]),
    "dlic_encode": (_I, [_VP, _IMGP, _I, C.POINTER(_I), _VP, _SZ, _VP, _VP, _VP, _SZ, _VP]),
    "dlic_encode_noalloc": (_I, [_VP, _IMGP, _I, C.POINTER(_I), _VP, _SZ, _VP, _VP, _VP]),
    "dlic_predict": (_I, [_VP, _IMGP, _I, _VP, _VP, _VP, _SZ, _VP]),
    "dlic_read_header": (_I, [_VP, _SZ, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I),
                              C.POINTER(C.c_uint64)]),
    "dlic_decode_workspace_size": (_I, [_VP, _IMGP, _I, C.POINTER(_SZ)]),
    "dlic_decode": (_I, [_VP, _VP, C.POINTER(C.c_uint64), _I, _IMGP, _VP, _VP, _SZ, _VP]),
    "dlic_encode_volume_workspace_size": (_I, [_VP, _VOLP, _I, C.POINTER(_SZ)]),
    "dlic_encode_volume": (_I, [_VP, _VOLP, _I, _VP, _SZ, _VP, _VP, _VP, _SZ, _VP]),
    "dlic_decode_volume_workspace_size": (_I, [_VP, _VOLP, _I, C.POINTER(_SZ)]),
    "dlic_decode_volume": (_I, [_VP, _VP, C.POINTER(C.c_uint64), _I, _VOLP, _VP, _VP, _SZ, _VP]),
    "dlic_train_param_count": (_SZ, [_I, _I, _I]),
    "dlic_trainer_create": (_I, [_I, _I, _I, _I, _I, _VP, C.POINTER(_VP)]),
    "dlic_train_param_count_k": (_SZ, [_I, _I, _I, _I]),
    "dlic_trainer_create_k": (_I, [_I, _I, _I, _I, _I, _I, _VP, C.POINTER(_VP)]),
    "dlic_trainer_destroy": (_I, [_VP]),
    "dlic_train_forward": (_I, [_VP, _VP, _VP, _I, _VP, _VP]),
    "dlic_train_backward": (_I, [_VP, _VP, _VP, _I, _VP, _VP, _VP]),
    "dlic_train_step": (_I, [_VP, _VP, _VP, _I, _VP, _VP]),
    "dlic_train_apply": (_I, [_VP, _VP, _VP]),
    "dlic_trainer_set_value_weights": (_I, [_VP, _VP]),
    "dlic_trainer_params": (_I, [_VP, _VP, _I, _VP]),
    "dlic_trainer_status": (_I, [_VP, C.POINTER(C.c_int32)]),
}


def lib():
    """The loaded library; raises if libdlic.so is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(code: int):
    if code != DLIC_OK:
        raise DlicError(code, (lib().dlic_last_error() or b"").decode())


def images_array(items):
    """items: iterable of (device_ptr, height, width, pitch)."""
    items = list(items)
    arr = (dlic_image * max(1, len(items)))()
    for i, (p, h, w, pitch) in enumerate(items):
        arr[i] = dlic_image(p, h, w, pitch)
    return arr, len(items)


def int_array(values):
    if values is None:
        return None
    values = list(values)
    return (C.c_int * max(1, len(values)))(*values)


def u64_array(values):
    values = list(values)
    return (C.c_uint64 * max(1, len(values)))(*values)


# --- thin wrappers, same names as the C ABI -------------------------------

def dlic_model_create(blob: bytes) -> int:
    buf = C.create_string_buffer(bytes(blob), len(blob))
    h = _VP()
    check(lib().dlic_model_create(buf, len(blob), C.byref(h)))
    return h.value


def dlic_model_destroy(model: int):
    check(lib().dlic_model_destroy(model))


def dlic_model_set_decode_plan(model: int, plan: int):
    check(lib().dlic_model_set_decode_plan(model, plan))


def dlic_model_set_peer_wait_limit(model: int, cycles: int):
    check(lib().dlic_model_set_peer_wait_limit(model, int(cycles)))


def dlic_model_info(model: int):
    p, h1, h2 = _I(), _I(), _I()
    hs = C.c_uint64()
    check(lib().dlic_model_info(model, C.byref(p), C.byref(h1), C.byref(h2), C.byref(hs)))
    return p.value, h1.value, h2.value, hs.value


def dlic_max_encoded_bytes(height: int, width: int, streams: int) -> int:
    return int(lib().dlic_max_encoded_bytes(height, width, streams))


def dlic_auto_streams(height: int, width: int) -> int:
    return int(lib().dlic_auto_streams(height, width))


def dlic_encode_workspace_size(model: int, images, streams=None) -> int:
    arr, n = images_array(images)
    out = _SZ()
    check(lib().dlic_encode_workspace_size(model, arr, n, int_array(streams), C.byref(out)))
    return out.value


def dlic_encode(model: int, images, streams, d_out: int, out_capacity: int, d_out_offsets: int,
                d_status: int, d_ws: int, ws_bytes: int, stream: int = 0):
    arr, n = images_array(images)
    check(lib().dlic_encode(model, arr, n, int_array(streams), d_out, out_capacity, d_out_offsets,
                            d_status or None, d_ws, ws_bytes, stream or None))


def dlic_predict(model: int, images, d_fc: int, d_status: int = 0, d_ws: int = 0, ws_bytes: int = 0,
                 stream: int = 0):
    arr, n = images_array(images)
    check(lib().dlic_predict(model, arr, n, d_fc, d_status or None, d_ws or None, ws_bytes, stream or None))


def dlic_encode_noalloc(model: int, images, streams, d_out: int, out_capacity: int,
                        d_out_offsets: int, d_status: int, stream: int = 0):
    """dlic_encode with the library's fixed scratch block as the workspace:
    for callers that cannot allocate device memory.  Calls share the block;
    do not let two of them overlap on the GPU."""
    arr, n = images_array(images)
    check(lib().dlic_encode_noalloc(model, arr, n, int_array(streams), d_out, out_capacity,
                                    d_out_offsets, d_status or None, stream or None))


def dlic_read_header(data: bytes):
    buf = C.create_string_buffer(bytes(data[:24]), 24) if len(data) >= 24 else C.create_string_buffer(bytes(data), max(1, len(data)))
    h, w, s, p = _I(), _I(), _I(), _I()
    hs = C.c_uint64()
    check(lib().dlic_read_header(buf, len(data), C.byref(h), C.byref(w), C.byref(s), C.byref(p),
                                 C.byref(hs)))
    return dict(height=h.value, width=w.value, streams=s.value, precision=p.value, hash=hs.value)


def dlic_decode_workspace_size(model: int, images) -> int:
    arr, n = images_array(images)
    out = _SZ()
    check(lib().dlic_decode_workspace_size(model, arr, n, C.byref(out)))
    return out.value


def dlic_decode(model: int, d_in: int, in_offsets, images, d_status: int, d_ws: int, ws_bytes: int,
                stream: int = 0):
    arr, n = images_array(images)
    check(lib().dlic_decode(model, d_in, u64_array(in_offsets), n, arr, d_status, d_ws, ws_bytes,
                            stream or None))


def volumes_array(volumes):
    """volumes: sequence of (ptr, depth, height, width, streams, pitch, slice_pitch)."""
    n = len(volumes)
    arr = (dlic_volume * max(1, n))()
    for i, v in enumerate(volumes):
        arr[i] = dlic_volume(*v)
    return arr, n


def dlic_encode_volume_workspace_size(model: int, volumes) -> int:
    arr, n = volumes_array(volumes)
    out = _SZ()
    check(lib().dlic_encode_volume_workspace_size(model, arr, n, C.byref(out)))
    return out.value


def dlic_encode_volume(model: int, volumes, d_out: int, out_capacity: int, d_out_offsets: int, d_status: int,
                       d_ws: int, ws_bytes: int, stream: int = 0):
    arr, n = volumes_array(volumes)
    check(lib().dlic_encode_volume(model, arr, n, d_out, out_capacity, d_out_offsets, d_status or None, d_ws,
                                   ws_bytes, stream or None))


def dlic_decode_volume_workspace_size(model: int, volumes) -> int:
    arr, n = volumes_array(volumes)
    out = _SZ()
    check(lib().dlic_decode_volume_workspace_size(model, arr, n, C.byref(out)))
    return out.value


def dlic_decode_volume(model: int, d_in: int, in_offsets, volumes, d_status: int, d_ws: int, ws_bytes: int,
                       stream: int = 0):
    arr, n = volumes_array(volumes)
    check(lib().dlic_decode_volume(model, d_in, u64_array(in_offsets), n, arr, d_status, d_ws, ws_bytes,
                                   stream or None))


def dlic_train_param_count(n_in: int, h1: int, h2: int) -> int:
    return int(lib().dlic_train_param_count(n_in, h1, h2))


def dlic_trainer_create(n_in: int, h1: int, h2: int, mode: int, max_batch: int, h_params) -> int:
    """h_params: contiguous float32 numpy array of dlic_train_param_count values."""
    h = _VP()
    check(lib().dlic_trainer_create(n_in, h1, h2, mode, max_batch, h_params.ctypes.data, C.byref(h)))
    return h.value


def dlic_train_param_count_k(n_in: int, h1: int, h2: int, n_out: int) -> int:
    return int(lib().dlic_train_param_count_k(n_in, h1, h2, n_out))


def dlic_trainer_create_k(n_in: int, h1: int, h2: int, n_out: int, mode: int, max_batch: int, h_params) -> int:
    """h_params: contiguous float32 numpy array of dlic_train_param_count_k values."""
    h = _VP()
    check(lib().dlic_trainer_create_k(n_in, h1, h2, n_out, mode, max_batch, h_params.ctypes.data, C.byref(h)))
    return h.value


def dlic_trainer_destroy(trainer: int):
    check(lib().dlic_trainer_destroy(trainer))


def dlic_train_forward(trainer: int, d_ctx: int, d_tgt: int, B: int, d_loss: int, stream: int = 0):
    check(lib().dlic_train_forward(trainer, d_ctx, d_tgt, B, d_loss, stream or None))


def dlic_train_backward(trainer: int, d_ctx: int, d_tgt: int, B: int, d_loss: int, d_grads: int,
                        stream: int = 0):
    check(lib().dlic_train_backward(trainer, d_ctx, d_tgt, B, d_loss, d_grads or None, stream or None))


def dlic_train_step(trainer: int, d_ctx: int, d_tgt: int, B: int, d_loss: int, stream: int = 0):
    check(lib().dlic_train_step(trainer, d_ctx, d_tgt, B, d_loss, stream or None))


def dlic_trainer_set_value_weights(trainer: int, weights=None, n_out: int = 256):
    """weights: one per target value, n_out of them (256, or 4096 for a
    12-bit trainer), or None for the plain loss."""
    if weights is None:
        check(lib().dlic_trainer_set_value_weights(trainer, None))
        return
    import numpy as np
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).reshape(-1))
    if w.size != n_out:
        raise ValueError(f"one weight per value ({n_out})")
    check(lib().dlic_trainer_set_value_weights(trainer, w.ctypes.data))


def dlic_train_apply(trainer: int, d_grads: int, stream: int = 0):
    check(lib().dlic_train_apply(trainer, d_grads, stream or None))


def dlic_trainer_params(trainer: int, d_params: int, write: bool, stream: int = 0):
    check(lib().dlic_trainer_params(trainer, d_params, int(bool(write)), stream or None))


def dlic_trainer_status(trainer: int) -> int:
    st = C.c_int32()
    check(lib().dlic_trainer_status(trainer, C.byref(st)))
    return st.value
