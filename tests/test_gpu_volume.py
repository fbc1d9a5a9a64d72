"""GPU parity for volumes coded with 3D windows (Sec. IV "3D Dependencies",
"3D Wavefront"): every slice's container from dlic_encode_volume must equal
the oracle's byte for byte, and dlic_decode_volume (all slices at once as a
3D wavefront) must return the volume."""
import numpy as np
import pytest
import torch

import synth
from paper_2207_05152_gb300 import model as M
from tests.helpers import calib_contexts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Codec():
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300.codec import Codec
    return Codec


def _blob(window, prec, h, vol, seed=3):
    layers = synth.predictive_mlp([M.window_size(window), h, h, 256], seed, window=window)
    if prec == "fp32":
        return M.fp32_blob(layers, window)
    return M.int8_blob(layers, calib_contexts(list(vol), window=window), window)


def _roundtrip(Codec, orc, blob, vols, streams, plan=0):
    from paper_2207_05152_gb300 import _lib
    codec = Codec(blob, decode_plan=plan)
    dev = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in vols]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out, offs = codec.encode_volume(dev, streams, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    offs = offs.cpu().tolist()
    host = out[:offs[-1]].cpu().numpy().tobytes()
    vol_offs, z0, S_used = [0], 0, []
    for v, s in zip(vols, streams):
        D, H, W = v.shape
        S = min(s or _lib.dlic_auto_streams(H, W), H)
        want, woffs = orc.encode_volume(blob, v, S)
        got = host[offs[z0]:offs[z0 + D]]
        assert [o - offs[z0] for o in offs[z0:z0 + D + 1]] == woffs
        assert got == want, f"volume {v.shape}: bitstream differs from the oracle"
        z0 += D
        vol_offs.append(offs[z0])
        S_used.append(S)
    data = out[:max(1, offs[-1])]
    dec, st = codec.decode_volume(data, vol_offs, [v.shape for v in vols], S_used)
    torch.cuda.synchronize()
    assert st[:len(vols)].cpu().tolist() == [0] * len(vols)
    for d, v in zip(dec, vols):
        assert np.array_equal(d.cpu().numpy(), v), f"volume {v.shape} decodes wrongly"
    codec.close()
    return host, offs


# (depth, height, width, streams): waves of a slice longer than the streams
# run on one cluster (sizes 1 to 16, the largest power of two dividing the
# streams), the others on the whole GPU (cooperative grid)
SHAPES = [(4, 40, 60, 16), (1, 9, 13, 3), (3, 1, 20, 1), (5, 7, 1, 4), (6, 33, 70, 8), (2, 64, 200, 32),
          (9, 40, 60, 20), (20, 96, 160, 64)]


@pytest.mark.parametrize("plan", ["auto", "image"])
@pytest.mark.parametrize("prec,h", [("int8", 128), ("fp32", 64)])
@pytest.mark.parametrize("window", [M.VOLUME_WINDOW, (2, 3, 1, 2, 2, 2, 2), (3, 2, 2, 0, 3, 1, 4)])
def test_volumes_match_oracle(Codec, orc, prec, h, window, plan):
    # plan "image" keeps every volume on one cluster
    from paper_2207_05152_gb300 import _lib
    vols = [synth.phantom_volume(d, hh, w, 13 * d + hh) for d, hh, w, _ in SHAPES]
    blob = _blob(window, prec, h, vols[0])
    code = _lib.DLIC_PLAN_AUTO if plan == "auto" else _lib.DLIC_PLAN_IMAGE
    for v, (_, _, _, s) in zip(vols, SHAPES):
        _roundtrip(Codec, orc, blob, [v], [s], code)


def test_volume_batch_and_auto_streams(Codec, orc):
    vols = [synth.phantom_volume(d, hh, w, 70 + d) for d, hh, w in [(7, 48, 64), (3, 100, 90), (12, 24, 40), (1, 30, 30)]]
    blob = _blob(M.VOLUME_WINDOW, "int8", 128, vols[0])
    _roundtrip(Codec, orc, blob, vols, [0, 0, 16, 0])


def test_volume_calls_refuse_2d_models_and_back(Codec):
    from paper_2207_05152_gb300 import _lib
    vol = synth.phantom_volume(2, 20, 30, 5)
    b3 = _blob(M.VOLUME_WINDOW, "int8", 128, vol)
    b2 = M.int8_blob(synth.predictive_mlp([12, 128, 128, 256], 3), calib_contexts([vol[0]]))
    c3, c2 = Codec(b3), Codec(b2)
    dv = torch.from_numpy(vol).cuda()
    with pytest.raises(_lib.DlicError) as e:
        c3.encode([dv[0]], [4])
    assert e.value.code == _lib.DLIC_ERR_INVALID
    with pytest.raises(_lib.DlicError) as e:
        c2.encode_volume([dv], [4])
    assert e.value.code == _lib.DLIC_ERR_INVALID
    c3.close()
    c2.close()


def test_corrupt_slice_is_reported(Codec, orc):
    from paper_2207_05152_gb300 import _lib
    vol = synth.phantom_volume(3, 24, 36, 8)
    blob = _blob(M.VOLUME_WINDOW, "int8", 128, vol)
    data, offs = orc.encode_volume(blob, vol, 8)
    codec = Codec(blob)
    # a later slice's window byte or model hash: the header check fails;
    # the last payload word: the volume must not come back as if intact
    for where, header in [(offs[1] + 12, True), (offs[2] + 16, True), (len(data) - 2, False)]:
        bad = bytearray(data)
        bad[where] ^= 0x41
        d = torch.frombuffer(bad, dtype=torch.uint8).cuda()
        dec, st = codec.decode_volume(d, [0, len(bad)], [vol.shape], [8])
        torch.cuda.synchronize()
        s = int(st[0].item())
        if header:
            assert s == _lib.DLIC_ERR_CORRUPT
        else:
            assert s == _lib.DLIC_ERR_CORRUPT or not np.array_equal(dec[0].cpu().numpy(), vol)
    codec.close()


def test_pitched_volume(Codec, orc):
    # rows and slices with padding: pitch > width, slice pitch > pitch x height,
    # read by the encoder and written by the decoder (grid and cluster paths)
    from paper_2207_05152_gb300 import _lib
    vol = synth.phantom_volume(5, 30, 44, 21)
    blob = _blob(M.VOLUME_WINDOW, "int8", 128, vol)
    for plan in (_lib.DLIC_PLAN_AUTO, _lib.DLIC_PLAN_IMAGE):
        codec = Codec(blob, decode_plan=plan)
        big = torch.zeros((5, 33, 52), dtype=torch.uint8, device="cuda")
        big[:, :30, :44] = torch.from_numpy(vol).cuda()
        view = big[:, :30, :44]
        out, offs = codec.encode_volume([view], [16])
        torch.cuda.synchronize()
        o = offs.cpu().tolist()
        want, woffs = orc.encode_volume(blob, vol, 16)
        assert out[:o[-1]].cpu().numpy().tobytes() == want
        dst = torch.full((5, 31, 47), 7, dtype=torch.uint8, device="cuda")
        dec, st = codec.decode_volume(out, [0, o[-1]], [vol.shape], [16], outs=[dst[:, :30, :44]])
        torch.cuda.synchronize()
        assert int(st[0].item()) == 0
        assert np.array_equal(dst[:, :30, :44].cpu().numpy(), vol)
        assert int(dst[:, 30:, :].max().item()) == 7 and int(dst[:, :, 44:].max().item()) == 7   # padding untouched
        codec.close()
