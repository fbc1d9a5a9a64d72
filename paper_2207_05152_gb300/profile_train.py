"""Runs a few training steps of one mode through the C ABI, for profilers.

    python -m paper_2207_05152_gb300.profile_train --mode bf16 --batch 65536 --steps 2
    python -m paper_2207_05152_gb300.profile_train --bits 12 --mode bf16x3 --batch 16384 --steps 2
    python -m paper_2207_05152_gb300.profile_train --mode bf16x3 --steps 2 --recompute

8-bit: 12-256-256-256 on contexts of eight 512 x 512 synthetic images;
12-bit: 12-128-128-4096 on contexts of twelve 256 x 256 12-bit phantoms.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="bf16", choices=["bf16", "bf16x3", "fp32"])
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--bits", type=int, default=8, choices=[8, 12])
    ap.add_argument("--recompute", action="store_true", help="activations recomputed rather than stored (BF16 modes)")
    args = ap.parse_args()
    import numpy as np
    import torch
    import synth
    from paper_2207_05152_gb300 import train as T
    if args.bits == 12:
        imgs = [synth.phantom_image12(256, 256, 1200 + i) for i in range(12)]
        widths = [12, 128, 128, 4096]
    else:
        imgs = [synth.config_image(3, i) for i in range(8)]
        widths = [12, 256, 256, 256]
    ctx, tgt = T.sample_contexts(imgs, args.batch, 3000)
    if args.bits == 12:
        ctx, tgt = ctx.view(np.int16), tgt.view(np.int16)
    tr = T.Trainer(synth.xavier_mlp(widths, 3), args.mode, max_batch=args.batch, recompute=args.recompute)
    c, t = torch.from_numpy(ctx).cuda(), torch.from_numpy(tgt).cuda()
    for _ in range(args.steps):
        tr.step(c, t)
    torch.cuda.synchronize()
    assert tr.status() == 0
    print("ok", args.mode, float(tr.loss.item()))


if __name__ == "__main__":
    main()
