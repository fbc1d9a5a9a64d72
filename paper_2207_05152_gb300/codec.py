"""PyTorch-facing wrapper of the C ABI: device buffers come from torch, work is
enqueued on torch's current CUDA stream, and every coding step runs in
libdlic.so."""
from __future__ import annotations

import torch

from . import _lib


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Codec:
    """One coder model on the current CUDA device (Sec. II-B: the same model
    and the same arithmetic at encode and decode).  Images are uint8 tensors
    for a model of 256 outputs; for a 12-bit model (4096 outputs, Sec. IV
    "Higher Bit Depth") they are int16 (or uint16) tensors of values
    0..4095, and decoded images come back as int16."""

    def __init__(self, blob: bytes, decode_plan: int = _lib.DLIC_PLAN_AUTO):
        if not torch.cuda.is_available():
            raise RuntimeError("the DLIC library needs a CUDA device")
        self.blob = bytes(blob)
        self.handle = _lib.dlic_model_create(self.blob)
        self.precision, self.h1, self.h2, self.hash = _lib.dlic_model_info(self.handle)
        from .model import model_symbols
        self.bits = 12 if model_symbols(self.blob) == 4096 else 8
        self.dtype = torch.int16 if self.bits == 12 else torch.uint8
        if decode_plan != _lib.DLIC_PLAN_AUTO:
            _lib.dlic_model_set_decode_plan(self.handle, decode_plan)
        self._ws = None

    def close(self):
        if self.handle:
            _lib.dlic_model_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _workspace(self, nbytes: int) -> torch.Tensor:
        nbytes = max(256, nbytes)
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        return self._ws

    def _desc(self, imgs):
        """(pointer, height, width, pitch in bytes) of each image."""
        ok = (torch.uint8,) if self.bits == 8 else (torch.int16, getattr(torch, "uint16", torch.int16))
        out = []
        for t in imgs:
            if t.dtype not in ok or t.dim() != 2 or not t.is_cuda:
                raise ValueError(f"images must be 2-D {'uint8' if self.bits == 8 else 'int16'} CUDA tensors")
            if t.stride(1) != 1:
                raise ValueError("image rows must be contiguous")
            out.append((t.data_ptr(), t.shape[0], t.shape[1], t.stride(0) * t.element_size()))
        return out

    def capacity(self, shapes, streams=None) -> int:
        streams = streams or [_lib.dlic_auto_streams(h, w) for h, w in shapes]
        return sum(_lib.dlic_max_encoded_bytes(h, w, s) for (h, w), s in zip(shapes, streams))

    def encode(self, images, streams=None, out=None, offsets=None, status=None, stream=None):
        """Encodes a list of 2-D uint8 CUDA tensors.  Returns (bytes tensor,
        offsets tensor of n + 1 int64 on the device); `status`, if given, is
        a 1-element int32 CUDA tensor that receives the device status."""
        desc = self._desc(images)
        shapes = [(d[1], d[2]) for d in desc]
        cap = self.capacity(shapes, streams)
        if out is None or out.numel() < cap:
            out = torch.empty(max(cap, 1), dtype=torch.uint8, device="cuda")
        if offsets is None:
            offsets = torch.empty(len(desc) + 1, dtype=torch.int64, device="cuda")
        ws_bytes = _lib.dlic_encode_workspace_size(self.handle, desc, streams)
        ws = self._workspace(ws_bytes)
        _lib.dlic_encode(self.handle, desc, streams, out.data_ptr(), out.numel(), offsets.data_ptr(),
                         status.data_ptr() if status is not None else 0, ws.data_ptr(), ws.numel(),
                         _stream_handle(stream))
        return out, offsets

    def predict(self, images, out=None, status=None, stream=None):
        """Per-pixel (f | c << 16) of every pixel's own value, raster order,
        images back to back (uint32 as an int32 CUDA tensor); `status`, if
        given, is a 1-element int32 CUDA tensor for the device status."""
        desc = self._desc(images)
        npx = sum(d[1] * d[2] for d in desc)
        if out is None or out.numel() < npx:
            out = torch.empty(max(npx, 1), dtype=torch.int32, device="cuda")
        ws = self._workspace(256)
        _lib.dlic_predict(self.handle, desc, out.data_ptr(), status.data_ptr() if status is not None else 0,
                          ws.data_ptr(), ws.numel(), _stream_handle(stream))
        return out

    def encode_to_bytes(self, images, streams=None):
        """Host bytes of each image's bitstream (synchronises)."""
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        out, offsets = self.encode(images, streams, status=status)
        if int(status.item()) != 0:
            raise _lib.DlicError(int(status.item()), "device status of dlic_encode")
        offs = offsets.cpu().tolist()
        host = out[: offs[-1]].cpu().numpy().tobytes()
        return [host[offs[i]:offs[i + 1]] for i in range(len(images))]

    def decode(self, data: torch.Tensor, offsets, shapes, outs=None, status=None, stream=None):
        """Decodes bitstreams held back to back in a uint8 CUDA tensor;
        offsets is a host sequence of n + 1 byte offsets.  Returns (list of
        decoded uint8 tensors, int32 status tensor on the device)."""
        n = len(shapes)
        if outs is None:
            outs = [torch.empty((h, w), dtype=self.dtype, device="cuda") for h, w in shapes]
        if status is None:
            status = torch.empty(max(1, n), dtype=torch.int32, device="cuda")
        desc = self._desc(outs)
        ws_bytes = _lib.dlic_decode_workspace_size(self.handle, desc)
        ws = self._workspace(ws_bytes)
        _lib.dlic_decode(self.handle, data.data_ptr(), [int(o) for o in offsets], desc,
                         status.data_ptr(), ws.data_ptr(), ws.numel(), _stream_handle(stream))
        return outs, status

    # --- volumes (3D window models; Sec. IV) ---

    @staticmethod
    def _vdesc(vols, streams):
        out = []
        for t, s in zip(vols, streams):
            if t.dtype != torch.uint8 or t.dim() != 3 or not t.is_cuda:
                raise ValueError("volumes must be 3-D uint8 CUDA tensors (depth, height, width)")
            if t.stride(2) != 1:
                raise ValueError("volume rows must be contiguous")
            out.append((t.data_ptr(), t.shape[0], t.shape[1], t.shape[2], int(s), t.stride(1), t.stride(0)))
        return out

    def encode_volume(self, volumes, streams=None, status=None, stream=None):
        """Encodes a list of (depth, height, width) uint8 CUDA tensors.
        Returns (bytes tensor, per-slice offsets tensor of sum(depth) + 1
        int64 on the device)."""
        streams = streams or [0] * len(volumes)
        desc = self._vdesc(volumes, streams)
        cap = 0
        for (_, d, h, w, s, _, _) in desc:
            cap += d * _lib.dlic_max_encoded_bytes(h, w, s or _lib.dlic_auto_streams(h, w))
        out = torch.empty(max(cap, 1), dtype=torch.uint8, device="cuda")
        offsets = torch.empty(sum(d[1] for d in desc) + 1, dtype=torch.int64, device="cuda")
        ws = self._workspace(_lib.dlic_encode_volume_workspace_size(self.handle, desc))
        _lib.dlic_encode_volume(self.handle, desc, out.data_ptr(), out.numel(), offsets.data_ptr(),
                                status.data_ptr() if status is not None else 0, ws.data_ptr(), ws.numel(),
                                _stream_handle(stream))
        return out, offsets

    def decode_volume(self, data: torch.Tensor, offsets, shapes, streams, outs=None, status=None, stream=None):
        """Decodes volumes; offsets: host sequence of n + 1 byte offsets (each
        volume's slice containers back to back); shapes: (depth, height,
        width) per volume; streams: each volume's stream count."""
        n = len(shapes)
        if outs is None:
            outs = [torch.empty(s, dtype=torch.uint8, device="cuda") for s in shapes]
        if status is None:
            status = torch.empty(max(1, n), dtype=torch.int32, device="cuda")
        desc = self._vdesc(outs, streams)
        ws = self._workspace(_lib.dlic_decode_volume_workspace_size(self.handle, desc))
        _lib.dlic_decode_volume(self.handle, data.data_ptr(), [int(o) for o in offsets], desc, status.data_ptr(),
                                ws.data_ptr(), ws.numel(), _stream_handle(stream))
        return outs, status

    def decode_bytes(self, streams_bytes, shapes=None):
        """Decodes host bitstreams; returns (list of host arrays, statuses):
        uint8 arrays, or uint16 arrays for a 12-bit model."""
        if shapes is None:
            shapes = []
            for b in streams_bytes:
                h = _lib.dlic_read_header(b)
                shapes.append((h["height"], h["width"]))
        offs = [0]
        for b in streams_bytes:
            offs.append(offs[-1] + len(b))
        data = torch.frombuffer(bytearray(b"".join(streams_bytes) or b"\0"), dtype=torch.uint8).cuda()
        outs, status = self.decode(data, offs, shapes)
        torch.cuda.synchronize()
        host = [o.cpu().numpy() for o in outs]
        if self.bits == 12:
            host = [h.view("<u2") for h in host]
        return host, status[: len(shapes)].cpu().tolist()
