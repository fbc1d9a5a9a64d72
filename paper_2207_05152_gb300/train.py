"""Training of the density network through the C ABI (dlic_train_*).

The loss is the categorical cross-entropy in bits, mean_b -log2 p(y_b | ctx_b)
(Sec. III-A reports it as "vloss in bpp").  `Trainer` owns the FP32 master
weights and Adam state on the device; `DlicLoss` exposes the hand-written
forward and backward kernels to torch.autograd (the gradient flows to a
parameter-sized tensor that stands for the trainer's weights).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from . import model as M

MODES = {"bf16": _lib.DLIC_TRAIN_BF16, "fp32": _lib.DLIC_TRAIN_FP32, "bf16x3": _lib.DLIC_TRAIN_BF16X3}
_DR = np.array([-2, -2, -2, -2, -2, -1, -1, -1, -1, -1, 0, 0])
_DC = np.array([-2, -1, 0, 1, 2, -2, -1, 0, 1, 2, -2, -1])


def flatten(layers) -> np.ndarray:
    """[(W1, b1), (W2, b2), (W3, b3)] -> the trainer's parameter vector."""
    return np.concatenate([np.asarray(a, np.float32).reshape(-1) for wb in layers for a in wb])


def unflatten(vec, h1: int, h2: int, n_in: int = 12, n_out: int = 256):
    v = np.asarray(vec, np.float32)
    shapes = [(h1, n_in), (h1,), (h2, h1), (h2,), (n_out, h2), (n_out,)]
    out, off = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(v[off:off + n].reshape(s))
        off += n
    return [(out[0], out[1]), (out[2], out[3]), (out[4], out[5])]


def _sample_dtype(images):
    """u16 for 12-bit images (Sec. IV "Higher Bit Depth"), else u8."""
    return np.uint16 if any(np.asarray(im).dtype == np.uint16 for im in images) else np.uint8


def _levels(images):
    return 4096 if _sample_dtype(images) == np.uint16 else 256


def sample_contexts(images, count: int, seed: int):
    """(ctx [count, 12], tgt [count]) at pixel positions drawn uniformly
    over the images; priors outside an image are 0 (the coder's window).
    u8 for 8-bit images, u16 for 12-bit ones.  Training-data preparation on
    the host; the coding path gathers on the device."""
    import synth
    idx, rr, cc = synth.sample_positions(images, count, seed)
    dt = _sample_dtype(images)
    ctx = np.zeros((count, 12), dt)
    tgt = np.zeros(count, dt)
    for i, img in enumerate(images):
        sel = np.nonzero(idx == i)[0]
        if sel.size == 0:
            continue
        H, W = img.shape
        pad = np.zeros((H + 2, W + 4), dt)
        pad[2:, 2:W + 2] = img
        r, c = rr[sel], cc[sel]
        ctx[sel] = pad[r[:, None] + 2 + _DR[None, :], c[:, None] + 2 + _DC[None, :]]
        tgt[sel] = img[r, c]
    return ctx, tgt


def sample_window_contexts(images, count: int, seed: int, window):
    """(ctx u8 [count, window size], tgt u8 [count]) for any causal window
    (u, l, r), or a 3D window (u, l, r, pu, pd, pl, pr) over the consecutive
    slices of a volume (`images` are then its slices; the lower layer comes
    from the slice before, zeros for the first).  Positions drawn uniformly;
    priors outside an image or the volume are 0."""
    import synth
    idx, rr, cc = synth.sample_positions(images, count, seed)
    return _contexts_at(images, idx, rr, cc, window)


def rare_value_positions(images, count: int, seed: int, alpha: float = 1.0):
    """`count` (image, row, col) triples drawn with probability proportional
    to hist(v)^-alpha, v the pixel's value and hist the value histogram over
    all the images (Sec. IV "Color Frequencies": rare values upsampled into
    the training set).  alpha = 1 draws every value present equally often;
    alpha = 0 is the uniform draw over pixels."""
    import synth
    flat = np.concatenate([im.reshape(-1) for im in images])
    hist = np.bincount(flat, minlength=_levels(images)).astype(np.float64)
    w = hist[flat] ** -float(alpha)
    cum = np.cumsum(w)
    u = synth.Rng(seed).uniform(count) * cum[-1]
    pick = np.minimum(np.searchsorted(cum, u, side="right"), flat.size - 1)
    sizes = np.array([im.size for im in images], dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    idx = np.searchsorted(starts, pick, side="right") - 1
    rem = pick - starts[idx]
    widths = np.array([im.shape[1] for im in images], dtype=np.int64)
    return idx, rem // widths[idx], rem % widths[idx]


def sample_upsampled_contexts(images, count: int, seed: int, window=M.DEFAULT_WINDOW, share: float = 0.25,
                              alpha: float = 1.0):
    """Training contexts with rare values upsampled (Sec. IV "Color
    Frequencies"): round(share * count) positions from rare_value_positions,
    the rest uniform (sample_window_contexts with the same seed), the
    upsampled ones last.  Drawing a context k times as often weights its
    loss term k-fold in expectation, so this one sampler also stands for the
    paper's frequency-weighted loss; share = 0 gives the uniform sampler's
    output exactly."""
    n_up = int(round(share * count))
    ctx, tgt = sample_window_contexts(images, count - n_up, seed, window)
    if n_up == 0:
        return ctx, tgt
    idx, rr, cc = rare_value_positions(images, n_up, seed + 0x5EED, alpha)
    c2, t2 = _contexts_at(images, idx, rr, cc, window)
    return np.concatenate([ctx, c2]), np.concatenate([tgt, t2])


def frequency_weights(images, alpha: float = 1.0):
    """Loss weights per value, hist(v)^-alpha normalised to mean 1 over the
    values present (absent values get 0): the frequency-weighted loss of
    Sec. IV "Color Frequencies", the counterpart of rare_value_positions.
    256 weights for 8-bit images, 4096 for 12-bit ones."""
    flat = np.concatenate([im.reshape(-1) for im in images])
    L = _levels(images)
    hist = np.bincount(flat, minlength=L).astype(np.float64)
    w = np.zeros(L)
    present = hist > 0
    w[present] = hist[present] ** -float(alpha)
    w[present] /= w[present].mean()
    return w.astype(np.float32)


def _contexts_at(images, idx, rr, cc, window):
    count = idx.size
    offs = M.window_offsets3(window)
    dt = _sample_dtype(images)
    ctx = np.zeros((count, len(offs)), dt)
    tgt = np.zeros(count, dt)
    for i, img in enumerate(images):
        sel = np.nonzero(idx == i)[0]
        if sel.size == 0:
            continue
        H, W = img.shape
        r, c = rr[sel], cc[sel]
        for k, (dz, dr, dc) in enumerate(offs):
            if i + dz < 0:
                continue
            src = images[i + dz]
            y, x = r + dr, c + dc
            ok = (y >= 0) & (y < H) & (x >= 0) & (x < W)
            ctx[sel[ok], k] = src[y[ok], x[ok]]
        tgt[sel] = img[r, c]
    return ctx, tgt


class Trainer:
    """FP32 master weights + Adam on the current CUDA device.  A network of
    4096 outputs (12-bit samples, Sec. IV "Higher Bit Depth") trains on u16
    contexts and targets; one of 256 on u8.  recompute (BF16 modes): two
    activation buffers instead of five, the first hidden layer recomputed in
    the backward pass; the results are bit for bit those without it."""

    def __init__(self, layers, mode: str = "bf16", max_batch: int = 65536, recompute: bool = False):
        self.n_in = layers[0][0].shape[1]   # the window's priors
        self.h1 = layers[0][0].shape[0]
        self.h2 = layers[1][0].shape[0]
        self.n_out = layers[2][0].shape[0]
        self.mode = mode
        self.nparams = _lib.dlic_train_param_count_k(self.n_in, self.h1, self.h2, self.n_out)
        flat = np.ascontiguousarray(flatten(layers))
        assert flat.size == self.nparams
        flags = _lib.DLIC_TRAIN_RECOMPUTE if recompute else 0
        self.handle = _lib.dlic_trainer_create_k(self.n_in, self.h1, self.h2, self.n_out, MODES[mode] | flags,
                                                 max_batch, flat)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def _check(self, ctx: torch.Tensor, tgt: torch.Tensor):
        want = torch.int16 if self.n_out == M.N_OUT_12 else torch.uint8
        for t in (ctx, tgt):
            if not (t.is_cuda and t.is_contiguous() and (t.dtype == want or (want == torch.int16 and
                                                                               t.dtype == torch.uint16))):
                raise ValueError(f"contexts and targets must be contiguous device tensors of "
                                 f"{'u16 samples' if want == torch.int16 else 'uint8'}")
        if ctx.numel() != tgt.numel() * self.n_in:
            raise ValueError("one context of n_in priors per target")

    def close(self):
        if self.handle:
            _lib.dlic_trainer_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream():
        return int(torch.cuda.current_stream().cuda_stream)

    def forward(self, ctx: torch.Tensor, tgt: torch.Tensor) -> torch.Tensor:
        self._check(ctx, tgt)
        _lib.dlic_train_forward(self.handle, ctx.data_ptr(), tgt.data_ptr(), tgt.numel(),
                                self.loss.data_ptr(), self._stream())
        return self.loss

    def backward(self, ctx: torch.Tensor, tgt: torch.Tensor, grads: torch.Tensor | None = None):
        if grads is None:
            grads = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        self._check(ctx, tgt)
        _lib.dlic_train_backward(self.handle, ctx.data_ptr(), tgt.data_ptr(), tgt.numel(),
                                 self.loss.data_ptr(), grads.data_ptr(), self._stream())
        return self.loss, grads

    def step(self, ctx: torch.Tensor, tgt: torch.Tensor) -> torch.Tensor:
        self._check(ctx, tgt)
        _lib.dlic_train_step(self.handle, ctx.data_ptr(), tgt.data_ptr(), tgt.numel(),
                             self.loss.data_ptr(), self._stream())
        return self.loss

    def set_value_weights(self, weights=None):
        """The frequency-weighted loss (Sec. IV "Color Frequencies"): one loss
        weight per target value (256, or 4096 for 12-bit samples), or None
        for the plain loss."""
        _lib.dlic_trainer_set_value_weights(self.handle, weights, self.n_out)

    def apply(self, grads: torch.Tensor):
        """One Adam update with the given gradient (device float32, the
        parameter layout): backward() then apply() of its own gradient is
        step()."""
        if grads.dtype != torch.float32 or not grads.is_cuda or grads.numel() != self.nparams:
            raise ValueError(f"grads must be {self.nparams} float32 values on the device")
        _lib.dlic_train_apply(self.handle, grads.contiguous().data_ptr(), self._stream())

    def params(self) -> torch.Tensor:
        out = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        _lib.dlic_trainer_params(self.handle, out.data_ptr(), False, self._stream())
        return out

    def set_params(self, flat: torch.Tensor):
        flat = flat.contiguous().float().cuda()
        _lib.dlic_trainer_params(self.handle, flat.data_ptr(), True, self._stream())

    def layers(self):
        return unflatten(self.params().cpu().numpy(), self.h1, self.h2, self.n_in, self.n_out)

    def fp32_blob(self, window=M.DEFAULT_WINDOW) -> bytes:
        """The trained network as an FP32 model blob for `window` (whose
        prior count is the trainer's n_in); a 12-bit network (4096
        outputs) takes the default window."""
        if self.n_out == M.N_OUT_12:
            return M.fp32_blob12(self.layers())
        return M.fp32_blob(self.layers(), window)

    def status(self) -> int:
        return _lib.dlic_trainer_status(self.handle)


class DlicLoss(torch.autograd.Function):
    """loss = DlicLoss.apply(theta, trainer, ctx, tgt): the bits loss of the
    trainer's network; theta is a parameter-sized tensor that receives the
    gradient (the kernels read the trainer's own master weights)."""

    @staticmethod
    def forward(fctx, theta, trainer, ctx, tgt):
        fctx.trainer = trainer
        fctx.save_for_backward(ctx, tgt)
        return trainer.forward(ctx, tgt).clone().reshape(())

    @staticmethod
    def backward(fctx, g):
        ctx, tgt = fctx.saved_tensors
        _, grads = fctx.trainer.backward(ctx, tgt)
        return grads * g, None, None, None
