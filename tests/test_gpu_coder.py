"""GPU parity: the CUDA coder against the oracle, bit for bit.

Bitstreams (header, word counts, every payload word) and decoded pixels must
be identical to the oracle's for the same seeded inputs (Sec. II-B
"Preprocessor": encoder and decoder must see the same network inputs and
produce the same PDFs; the image is reproduced losslessly)."""
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


def _models(widths, seed, images):
    layers = synth.predictive_mlp(widths, seed)
    return {"fp32": M.fp32_blob(layers), "int8": M.int8_blob(layers, calib_contexts(images))}


def _check(Codec, orc, blob, imgs, streams, plan=0):
    codec = Codec(blob, decode_plan=plan)
    got = codec.encode_to_bytes([torch.from_numpy(np.ascontiguousarray(i)).cuda() for i in imgs], streams)
    for k, img in enumerate(imgs):
        from paper_2207_05152_gb300 import _lib
        S = streams[k] if streams else _lib.dlic_auto_streams(img.shape[0], img.shape[1])
        want = orc.encode(blob, img, S)
        assert got[k] == want, f"image {k}: bitstream differs from the oracle"
    dec, status = codec.decode_bytes(got)
    assert status == [0] * len(imgs)
    for k, img in enumerate(imgs):
        assert np.array_equal(dec[k], img)
    codec.close()
    return got


def test_cfg1_fp32_64x64_s32(Codec, orc):
    img = synth.config_image(1)
    blob = M.fp32_blob(synth.predictive_mlp([12, 64, 64, 256], 1))
    _check(Codec, orc, blob, [img], [32])


@pytest.mark.parametrize("prec", ["int8", "fp32"])
def test_cfg2_512x512_s256(Codec, orc, prec):
    img = synth.config_image(2)
    blob = _models([12, 128, 128, 256], 2, [img])[prec]
    _check(Codec, orc, blob, [img], [256])


SHAPES = [(1, 1, 1), (1, 7, 1), (7, 1, 4), (2, 3, 2), (5, 64, 9), (16, 16, 16), (13, 40, 3),
          (9, 50, 1), (33, 17, 32), (3, 200, 2), (70, 130, 70), (80, 250, 7)]


@pytest.mark.parametrize("prec,widths", [("fp32", [12, 32, 48, 256]), ("int8", [12, 32, 48, 256]),
                                         ("int8", [12, 128, 128, 256]), ("fp32", [12, 32, 256, 256])])
def test_edge_shapes(Codec, orc, prec, widths):
    # INT8 12-128-128-256 runs the tensor-core encoder and the cluster
    # wavefront decoder; the narrower INT8 network the tensor-core encoder and
    # the one-CTA-per-image decoder; FP32 with h2 <= 128 the CUDA-core encoder
    # and the FP32 cluster wavefront decoder; FP32 with h2 = 256 the
    # one-CTA-per-image decoder.
    imgs = [synth.value_noise_image(h, w, 7 * h + w) for h, w, _ in SHAPES]
    blob = _models(widths, 5, [synth.voronoi_image(40, 40, 2)])[prec]
    _check(Codec, orc, blob, imgs, [s for _, _, s in SHAPES])


def test_auto_streams_and_batch(Codec, orc):
    imgs = synth.batch_images(6, 31, hmin=20, hmax=90, wmin=30, wmax=160)
    blob = _models([12, 128, 128, 256], 3, imgs[:2])["int8"]
    _check(Codec, orc, blob, imgs, None)


def test_pitched_image(Codec, orc):
    img = synth.voronoi_image(40, 50, 3)
    blob = _models([12, 64, 64, 256], 4, [img])["int8"]
    codec = Codec(blob)
    big = torch.zeros((40, 64), dtype=torch.uint8, device="cuda")
    big[:, :50] = torch.from_numpy(img).cuda()
    got = codec.encode_to_bytes([big[:, :50]], [8])[0]
    assert got == orc.encode(blob, img, 8)
    codec.close()


@pytest.mark.parametrize("prec,widths", [("fp32", [12, 32, 32, 256]), ("int8", [12, 128, 128, 256])])
def test_corrupt_and_capacity(Codec, orc, prec, widths):
    from paper_2207_05152_gb300 import _lib
    img = synth.value_noise_image(20, 30, 2)
    blob = _models(widths, 6, [img])[prec]
    codec = Codec(blob)
    data = bytearray(orc.encode(blob, img, 4))
    _, st = codec.decode_bytes([bytes(data[:-2])], [(20, 30)])
    assert st == [_lib.DLIC_ERR_CORRUPT]
    bad = bytearray(data)
    bad[16] ^= 1                                   # model hash
    _, st = codec.decode_bytes([bytes(bad)], [(20, 30)])
    assert st == [_lib.DLIC_ERR_CORRUPT]
    bad = bytearray(data)
    bad[24 + 16] ^= 0x80                           # first flush word of stream 0
    dec, st = codec.decode_bytes([bytes(bad)], [(20, 30)])
    assert st == [_lib.DLIC_ERR_CORRUPT] or not np.array_equal(dec[0], img)
    want_status, want_img = orc.decode(blob, bytes(bad), 20, 30)
    assert (st[0] == 0) == (want_status == 0)
    t = torch.from_numpy(img).cuda()
    out = torch.empty(16, dtype=torch.uint8, device="cuda")
    offs = torch.empty(2, dtype=torch.int64, device="cuda")
    ws = codec._workspace(1 << 20)
    with pytest.raises(_lib.DlicError) as e:
        _lib.dlic_encode(codec.handle, codec._desc([t]), [4], out.data_ptr(), out.numel(),
                         offs.data_ptr(), 0, ws.data_ptr(), ws.numel(), 0)
    assert e.value.code == _lib.DLIC_ERR_CAPACITY
    codec.close()


@pytest.mark.parametrize("prec,widths,plan", [("int8", [12, 32, 32, 256], 0), ("int8", [12, 128, 128, 256], 0),
                                              ("int8", [12, 128, 128, 256], 3), ("fp32", [12, 64, 64, 256], 1)])
def test_word_counts_that_wrap_32_bits_are_corrupt(Codec, orc, prec, widths, plan):
    # 1030 streams, more than one per decoder thread: two counts of the same
    # thread raised by 2^31 each leave a 32-bit sum (and so the total-length
    # check) unchanged, but would put the next stream's start 2^31 words past
    # the input.  Every decoder must report a corrupt stream instead.
    from paper_2207_05152_gb300 import _lib
    H, W, S = 1030, 5, 1030
    img = synth.value_noise_image(H, W, 41)
    blob = _models(widths, 6, [synth.voronoi_image(40, 40, 2)])[prec]
    data = bytearray(orc.encode(blob, img, S))
    for s in (0, 1):
        c = int.from_bytes(data[24 + 4 * s:28 + 4 * s], "little")
        data[24 + 4 * s:28 + 4 * s] = (c + (1 << 31)).to_bytes(4, "little")
    want_status, _ = orc.decode(blob, bytes(data), H, W)
    assert want_status == _lib.DLIC_ERR_CORRUPT
    codec = Codec(blob, decode_plan=plan)
    _, st = codec.decode_bytes([bytes(data)], [(H, W)])
    assert st == [_lib.DLIC_ERR_CORRUPT]
    codec.close()


def test_batched_decode_mixed_cluster_sizes(Codec, orc):
    # Twelve images of different sizes in one call: the autotuner gives them
    # different cluster sizes, which run as concurrent groups.
    sizes = [(30, 40), (64, 64), (100, 180), (20, 300), (150, 90), (200, 260), (45, 45), (120, 400),
             (16, 16), (90, 120), (300, 200), (60, 500)]
    imgs = [synth.voronoi_image(h, w, 500 + i) for i, (h, w) in enumerate(sizes)]
    blob = _models([12, 128, 128, 256], 8, imgs[:3])["int8"]
    _check(Codec, orc, blob, imgs, None)


def test_wide_images_small_clusters(Codec, orc):
    # wide images among many small ones get small clusters: hundreds of
    # pixels per CTA and wave, large rings, smaller pixel chunks
    sizes = [(40, 2048), (300, 1600)] + [(24, 32)] * 40
    imgs = [synth.voronoi_image(h, w, 900 + i) for i, (h, w) in enumerate(sizes)]
    blob = _models([12, 128, 128, 256], 11, imgs[:1])["int8"]
    _check(Codec, orc, blob, imgs, None)


def test_fp32_batched_decode_mixed_cluster_sizes(Codec, orc):
    # The FP32 cluster decoder over a batch of uneven sizes (cluster sizes
    # from 1 upwards, several chunks of pixels per wave in the small clusters).
    sizes = [(24, 40), (70, 90), (130, 250), (18, 200), (160, 60), (40, 320)]
    imgs = [synth.voronoi_image(h, w, 700 + i) for i, (h, w) in enumerate(sizes)]
    blob = _models([12, 64, 64, 256], 10, imgs[:2])["fp32"]
    _check(Codec, orc, blob, imgs, None)


def test_decode_inside_cuda_graph(Codec, orc):
    img = synth.voronoi_image(96, 160, 21)
    blob = _models([12, 128, 128, 256], 9, [img])["int8"]
    codec = Codec(blob)
    d_img = torch.from_numpy(img).cuda()
    out, offs = codec.encode([d_img], None)
    torch.cuda.synchronize()
    o = offs.cpu().tolist()
    dec = torch.empty_like(d_img)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    codec.decode(out, o, [img.shape], outs=[dec], status=status)   # warm-up outside capture
    torch.cuda.synchronize()
    dec.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        codec.decode(out, o, [img.shape], outs=[dec], status=status)
    g.replay()
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and torch.equal(dec, d_img)
    codec.close()


# --- other causal windows ("any window shape", Sec. II-A; Fig. 6's 9 x 9) ---

def _window_models(widths, seed, images, window):
    from tests.helpers import calib_contexts
    layers = synth.predictive_mlp(widths, seed, window=window)
    return {"fp32": M.fp32_blob(layers, window),
            "int8": M.int8_blob(layers, calib_contexts(images, window=window), window)}


@pytest.mark.parametrize("window", [M.FIG6_WINDOW, (4, 1, 2), (1, 3, 2), (3, 1, 1), (1, 7, 1)])
@pytest.mark.parametrize("prec,h", [("int8", 128), ("fp32", 64)])
def test_windows_match_oracle(Codec, orc, window, prec, h):
    # tensor-core INT8 encoder and cluster decoder (first-layer K = the
    # window's priors padded to 16; rings with one slot per row distance),
    # FP32 tiled encoder and FP32 cluster decoder
    n = M.window_size(window)
    shapes = [(96, 160, 16), (1, 9, 1), (7, 1, 4), (20, 33, 5), (40, 260, 8)]
    imgs = [synth.voronoi_image(hh, ww, 11 * hh + ww) for hh, ww, _ in shapes]
    blob = _window_models([n, h, h, 256], 12, imgs[:1], window)[prec]
    got = _check(Codec, orc, blob, imgs, [s for _, _, s in shapes])
    assert all(g[12] == window[0] for g in got)


def test_fig6_window_batched_cluster_sizes(Codec, orc):
    # cluster sizes from 1 (byte ring, one cluster barrier per wave) to 16
    sizes = [(30, 40), (200, 260), (16, 16), (120, 400), (300, 200), (60, 500)]
    imgs = [synth.voronoi_image(hh, ww, 950 + i) for i, (hh, ww) in enumerate(sizes)]
    blob = _window_models([78, 128, 128, 256], 13, imgs[:1], M.FIG6_WINDOW)["int8"]
    _check(Codec, orc, blob, imgs, None)


def test_window_needs_supported_kernels(Codec):
    from paper_2207_05152_gb300 import _lib
    img = synth.voronoi_image(40, 40, 2)
    blob = _window_models([78, 64, 64, 256], 14, [img], M.FIG6_WINDOW)["int8"]   # INT8 decode needs 128/128
    with pytest.raises(_lib.DlicError) as e:
        Codec(blob)
    assert e.value.code == _lib.DLIC_ERR_UNSUPPORTED


# --- decoder prior plans (tagged ring, byte ring, read back from the image) ---

@pytest.mark.parametrize("plan", ["byte_ring", "image"])
@pytest.mark.parametrize("prec,h,window", [("int8", 128, M.DEFAULT_WINDOW), ("fp32", 64, M.DEFAULT_WINDOW),
                                           ("int8", 128, M.FIG6_WINDOW), ("fp32", 64, M.FIG6_WINDOW)])
def test_forced_decode_plans(Codec, orc, plan, prec, h, window):
    # every plan decodes the same pixels; cluster sizes 1 to 16 over the batch
    from paper_2207_05152_gb300 import _lib
    sizes = [(96, 160), (1, 9), (7, 1), (20, 33), (200, 260), (120, 400), (300, 200), (16, 16)]
    imgs = [synth.voronoi_image(hh, ww, 31 * hh + ww) for hh, ww in sizes]
    blob = _window_models([M.window_size(window), h, h, 256], 15, imgs[:1], window)[prec]
    code = {"byte_ring": _lib.DLIC_PLAN_BYTE_RING, "image": _lib.DLIC_PLAN_IMAGE}[plan]
    codec = Codec(blob, decode_plan=code)
    dev = [torch.from_numpy(i).cuda() for i in imgs]
    got = codec.encode_to_bytes(dev, None)
    for k, img in enumerate(imgs):
        assert got[k] == orc.encode(blob, img, _lib.dlic_auto_streams(*img.shape))
    dec, status = codec.decode_bytes(got)
    assert status == [0] * len(imgs)
    for k, img in enumerate(imgs):
        assert np.array_equal(dec[k], img), f"image {k} {img.shape}"
    codec.close()


def test_long_waves_read_priors_from_image():
    # 4096 x 12288: waves of 4096 pixels are too long for the rings, so the
    # cluster decoder reads priors back from the output image; the round trip
    # must be lossless (a property that holds at any size)
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300.codec import Codec as C
    tile = synth.voronoi_image(512, 768, 77)
    img = np.ascontiguousarray(np.tile(tile, (8, 16)))
    img[::7, ::5] ^= 0x55                     # break the tiling's periodicity
    blob = _models([12, 128, 128, 256], 16, [tile])["int8"]
    codec = C(blob)
    d = torch.from_numpy(img).cuda()
    out, offs = codec.encode([d], None)
    o = offs.cpu().tolist()
    dec = torch.empty_like(d)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    codec.decode(out, o, [img.shape], outs=[dec], status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and torch.equal(dec, d)
    codec.close()


def test_waves_beyond_every_plan_are_refused(Codec):
    # 30000 x 90000: no shared-memory plan holds a wave's rows; the call
    # fails on the host before anything is enqueued (the buffers are real
    # and large enough all the same)
    from paper_2207_05152_gb300 import _lib
    blob = _models([12, 128, 128, 256], 17, [synth.voronoi_image(40, 40, 3)])["int8"]
    codec = Codec(blob)
    H, W = 30000, 90000
    out = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    data = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = codec._workspace(_lib.dlic_decode_workspace_size(codec.handle, codec._desc([out])))
    with pytest.raises(_lib.DlicError) as e:
        _lib.dlic_decode(codec.handle, data.data_ptr(), [0, data.numel()], codec._desc([out]), st.data_ptr(),
                         ws.data_ptr(), ws.numel(), 0)
    assert e.value.code == _lib.DLIC_ERR_UNSUPPORTED
    codec.close()
    del out
    torch.cuda.empty_cache()


# --- the grid decoder: a batch's waves over every SM (cooperative launch) ---

@pytest.mark.parametrize("prec,widths", [("int8", [12, 128, 128, 256]), ("fp32", [12, 64, 64, 256])])
def test_grid_plan_edge_shapes(Codec, orc, prec, widths):
    # images whose waves hold two rows of one stream (streams below the wave
    # length) go whole to one CTA per wave, the others are split evenly
    from paper_2207_05152_gb300 import _lib
    imgs = [synth.value_noise_image(h, w, 7 * h + w) for h, w, _ in SHAPES]
    blob = _models(widths, 5, [synth.voronoi_image(40, 40, 2)])[prec]
    _check(Codec, orc, blob, imgs, [s for _, _, s in SHAPES], _lib.DLIC_PLAN_GRID)


@pytest.mark.parametrize("window", [M.DEFAULT_WINDOW, M.FIG6_WINDOW])
def test_grid_plan_batch(Codec, orc, window):
    from paper_2207_05152_gb300 import _lib
    sizes = [(30, 40), (64, 64), (100, 180), (20, 300), (150, 90), (200, 260), (45, 45), (120, 400),
             (16, 16), (90, 120), (300, 200), (60, 500)]
    imgs = [synth.voronoi_image(h, w, 800 + i) for i, (h, w) in enumerate(sizes)]
    blob = _window_models([M.window_size(window), 128, 128, 256], 8, imgs[:3], window)["int8"]
    _check(Codec, orc, blob, imgs, None, _lib.DLIC_PLAN_GRID)


def test_auto_plan_takes_the_grid_for_very_wide_images():
    # one 1100 x 3300 image: waves of 1100 pixels, more than 64 for each CTA
    # of a 16-CTA cluster, so the automatic plan takes the grid; the round
    # trip must be lossless (the encoder is pinned to the oracle elsewhere)
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300.codec import Codec as C
    tile = synth.voronoi_image(550, 660, 31)
    img = np.ascontiguousarray(np.tile(tile, (2, 5)))
    img[::5, ::3] ^= 0x33
    blob = _models([12, 128, 128, 256], 9, [tile])["int8"]
    codec = C(blob)
    d = torch.from_numpy(img).cuda()
    out, offs = codec.encode([d], None)
    o = offs.cpu().tolist()
    dec = torch.empty_like(d)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    codec.decode(out, o, [img.shape], outs=[dec], status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and torch.equal(dec, d)
    codec.close()
