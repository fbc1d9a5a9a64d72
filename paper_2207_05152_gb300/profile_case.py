"""Runs a named workload a few times through the C ABI, for profilers.

    python -m paper_2207_05152_gb300.profile_case --case cfg2 --iters 2
    python -m paper_2207_05152_gb300.profile_case --case cfg4 --count 8 --iters 1
    python -m paper_2207_05152_gb300.profile_case --case volume --iters 1
    python -m paper_2207_05152_gb300.profile_case --case deep --size 128 --iters 1
    python -m paper_2207_05152_gb300.profile_case --case twelve --size 64 --iters 1
    python -m paper_2207_05152_gb300.profile_case --case wide --size 64 --iters 1

Each iteration encodes and decodes the batch and checks the round trip.
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
    ap.add_argument("--case", default="cfg2", choices=["cfg2", "cfg4", "volume", "deep", "twelve", "wide"])
    ap.add_argument("--size", type=int, default=128, help="deep / twelve: the square image's side")
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--count", type=int, default=8)
    ap.add_argument("--precision", default="int8", choices=["int8", "fp32"])
    args = ap.parse_args()
    import torch
    from paper_2207_05152_gb300 import workloads
    from paper_2207_05152_gb300.codec import Codec
    if args.case == "volume":
        # the 35 x 256 x 256 scan with the 3D window (grid decoder)
        from paper_2207_05152_gb300 import _lib, model as M
        _, b3, b3f = workloads.models(window=M.VOLUME_WINDOW)
        vol = workloads.volume_scan()
        codec = Codec(b3 if args.precision == "int8" else b3f)
        dv = torch.from_numpy(vol).cuda()
        S = _lib.dlic_auto_streams(vol.shape[1], vol.shape[2])
        for _ in range(args.iters):
            out, offs = codec.encode_volume([dv], [S])
            o = offs.cpu().tolist()
            dec, status = codec.decode_volume(out, [0, o[-1]], [vol.shape], [S])
            torch.cuda.synchronize()
            assert int(status[0].item()) == 0 and torch.equal(dec[0], dv)
        print("ok volume", vol.shape)
        return
    if args.case == "wide":
        # two hidden layers of 4096 units on a square crop of the cfg-2 image
        import numpy as np
        w8, w32 = workloads.wide_models()
        codec = Codec(w8 if args.precision == "int8" else w32)
        img = np.ascontiguousarray(workloads.cfg2_image()[:args.size, :args.size])
        dv = torch.from_numpy(img).cuda()
        for _ in range(args.iters):
            out, offs = codec.encode([dv], [min(args.size, 64)])
            o = offs.cpu().tolist()
            dec, status = codec.decode(out, o, [img.shape])
            torch.cuda.synchronize()
            assert int(status[0].item()) == 0 and torch.equal(dec[0], dv)
        print("ok wide", img.shape)
        return
    if args.case in ("deep", "twelve"):
        # six dense layers (five hidden, widths 128) on an 8-bit crop of the
        # cfg-2 image, or a 12-bit MRI-like slice with 12-128-128-4096
        import numpy as np
        import synth
        from paper_2207_05152_gb300 import model as M
        n = args.size
        if args.case == "deep":
            deep8, deep32 = workloads.deep_models()
            codec = Codec(deep8 if args.precision == "int8" else deep32)
            img = np.ascontiguousarray(workloads.cfg2_image()[:n, :n])
            dv = torch.from_numpy(img).cuda()
        else:
            codec = Codec(M.fp32_blob12(synth.predictive_mlp([12, 128, 128, 4096], 12, sigma=96.0, levels=4096)))
            img = synth.phantom_image12(n, n, 12)
            dv = torch.from_numpy(img.astype(np.int16)).cuda()
        for _ in range(args.iters):
            out, offs = codec.encode([dv], [min(n, 96)])
            o = offs.cpu().tolist()
            dec, status = codec.decode(out, o, [img.shape])
            torch.cuda.synchronize()
            assert int(status[0].item()) == 0 and torch.equal(dec[0], dv)
        print("ok", args.case, img.shape)
        return
    _, blob8, blob32 = workloads.models()
    imgs = [workloads.cfg2_image()] if args.case == "cfg2" else workloads.cfg4_images(args.count)
    streams = [256] if args.case == "cfg2" else None
    codec = Codec(blob8 if args.precision == "int8" else blob32)
    dev = [torch.from_numpy(i).cuda() for i in imgs]
    shapes = [i.shape for i in imgs]
    for _ in range(args.iters):
        out, offs = codec.encode(dev, streams)
        o = offs.cpu().tolist()
        dec, status = codec.decode(out, o, shapes)
        torch.cuda.synchronize()
        assert status[: len(imgs)].cpu().tolist() == [0] * len(imgs)
        assert all(torch.equal(a, b) for a, b in zip(dec, dev))
    print("ok", args.case, len(imgs), "images")


if __name__ == "__main__":
    main()
