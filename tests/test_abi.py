"""The C-ABI library builds, loads without a GPU and exports every entry point
include/dlic.h declares; host-side argument checks run without a device."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"DLIC_API\s+[\w\s\*]+?\b(dlic_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2207_05152_gb300 import build
    build.build()
    from paper_2207_05152_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 11
    L = lib.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names <= set(lib.SIGNATURES), names - set(lib.SIGNATURES)


def test_host_side_helpers(lib):
    assert lib.dlic_max_encoded_bytes(64, 64, 32) == 24 + 4 * 32 + 2 * (4096 + 64)
    assert lib.dlic_max_encoded_bytes(3, 10, 99) == 24 + 4 * 3 + 2 * (30 + 6)
    assert lib.dlic_auto_streams(512, 512) == 176
    assert lib.dlic_auto_streams(100, 2048) == 100
    assert lib.dlic_auto_streams(64, 64) == 32
    assert lib.dlic_auto_streams(5, 64) == 5


def test_header_parser_and_model_checks(lib, orc):
    import synth
    from paper_2207_05152_gb300 import model as M
    blob = M.fp32_blob(synth.predictive_mlp([12, 32, 32, 256], 1))
    img = synth.value_noise_image(10, 20, 1)
    data = orc.encode(blob, img, 4)
    h = lib.dlic_read_header(data)
    assert (h["height"], h["width"], h["streams"], h["precision"]) == (10, 20, 4, 0)
    assert h["hash"] == orc.fnv1a64(blob)
    with pytest.raises(lib.DlicError) as e:
        lib.dlic_read_header(b"XXXX" + data[4:])
    assert e.value.code == lib.DLIC_ERR_CORRUPT
    # malformed blobs are rejected on the host before any device work
    with pytest.raises(lib.DlicError) as e:
        lib.dlic_model_create(blob[:-4])
    assert e.value.code == lib.DLIC_ERR_INVALID
    bad = bytearray(blob)
    bad[32:36] = (5).to_bytes(4, "little")   # lut[0] must be 2^23
    with pytest.raises(lib.DlicError) as e:
        lib.dlic_model_create(bytes(bad))
    assert e.value.code == lib.DLIC_ERR_INVALID


def test_window_contexts_match_the_default_sampler():
    import numpy as np
    # the general sampler with the default window gives the 12-prior contexts
    import synth
    from paper_2207_05152_gb300 import train as T
    imgs = [synth.voronoi_image(30, 41, 5), synth.voronoi_image(17, 9, 6)]
    a, ta = T.sample_contexts(imgs, 500, 3)
    b, tb = T.sample_window_contexts(imgs, 500, 3, (2, 2, 2))
    assert np.array_equal(a, b) and np.array_equal(ta, tb)


def test_deeper_network_blobs_are_checked_before_any_device_call(lib):
    # "DLM2" blobs the GPU library refuses while parsing (no device needed):
    # another window with other than two hidden layers, hidden widths outside
    # the one-pixel-per-thread kernels' range, malformed headers
    import struct
    import synth
    from paper_2207_05152_gb300 import model as M

    def deep(widths, window=M.DEFAULT_WINDOW, seed=5):
        rng = synth.Rng(seed)
        dims = [M.window_size(window)] + widths + [256]
        layers = [((0.1 * rng.normal(o * i)).reshape(o, i).astype(np.float32), np.zeros(o, np.float32))
                  for i, o in zip(dims[:-1], dims[1:])]
        return M.deep_fp32_blob(layers, window)

    cases = [
        (deep([32, 32, 32], window=(3, 3, 2)), lib.DLIC_ERR_UNSUPPORTED),   # three hidden layers, wider window
        (deep([32, 6, 32]), lib.DLIC_ERR_UNSUPPORTED),                      # width not a multiple of 4
        (deep([32, 258, 32]), lib.DLIC_ERR_UNSUPPORTED),                    # wider than 256, not a multiple of 4
        (deep([300, 40], window=(3, 3, 2)), lib.DLIC_ERR_UNSUPPORTED),      # wider than 256, wider window
        (deep([24, 40]), lib.DLIC_ERR_UNSUPPORTED),                         # two hidden layers: multiples of 16
    ]
    good = deep([32, 48, 32])
    too_wide = bytearray(good)
    too_wide[20:24] = struct.pack("<I", 4100)                               # the second width above 4096
    cases.append((bytes(too_wide), lib.DLIC_ERR_INVALID))
    bad_l = bytearray(good)
    bad_l[12:16] = struct.pack("<I", 0)                                      # no hidden layer
    cases.append((bytes(bad_l), lib.DLIC_ERR_INVALID))
    bad_w = bytearray(good)
    bad_w[28:32] = struct.pack("<I", 16)                                     # a width past L
    cases.append((bytes(bad_w), lib.DLIC_ERR_INVALID))
    cases.append((good[:-4], lib.DLIC_ERR_INVALID))                          # truncated
    cases.append((good + b"\0\0\0\0", lib.DLIC_ERR_INVALID))                # trailing bytes
    for blob, code in cases:
        with pytest.raises(lib.DlicError) as e:
            lib.dlic_model_create(blob)
        assert e.value.code == code, (len(blob), e.value)


def test_twelve_bit_blobs_are_checked_before_any_device_call(lib):
    # 4096 outputs (12-bit pixels): FP32 only, the default window, hidden
    # widths multiples of 4 up to 256
    import struct
    import synth
    from paper_2207_05152_gb300 import model as M

    def net(widths, window=M.DEFAULT_WINDOW, seed=6):
        rng = synth.Rng(seed)
        dims = [M.window_size(window)] + widths + [4096]
        return [((0.1 * rng.normal(o * i)).reshape(o, i).astype(np.float32), np.zeros(o, np.float32))
                for i, o in zip(dims[:-1], dims[1:])]

    i8 = [M._header(M.PREC_INT8, 32, 32, M.DEFAULT_WINDOW, 4096)]
    for o, i in ((32, 12), (32, 32), (4096, 32)):
        i8 += [np.zeros((o, i), np.int8).tobytes(), np.ones(o, "<f4").tobytes(), np.zeros(o, "<f4").tobytes()]
    cases = [
        (b"".join(i8), lib.DLIC_ERR_INVALID),                                        # INT8, 4096 outputs
        (M.deep_fp32_blob(net([32, 32], (3, 3, 2)), (3, 3, 2)), lib.DLIC_ERR_UNSUPPORTED),   # another window
        (M.deep_fp32_blob(net([32, 6])), lib.DLIC_ERR_UNSUPPORTED),                 # width not a multiple of 4
        (M.deep_fp32_blob(net([32, 512])), lib.DLIC_ERR_UNSUPPORTED),               # width above 256
    ]
    good = M.fp32_blob12(net([32, 32]))
    bad_out = bytearray(good)
    bad_out[20:24] = struct.pack("<I", 1024)                                         # neither 256 nor 4096
    cases.append((bytes(bad_out), lib.DLIC_ERR_INVALID))
    cases.append((good[:-4], lib.DLIC_ERR_INVALID))
    for blob, code in cases:
        with pytest.raises(lib.DlicError) as e:
            lib.dlic_model_create(blob)
        assert e.value.code == code, (len(blob), e.value)


def test_read_header_of_a_twelve_bit_container(lib, orc):
    # the host-side header parse: byte 13 carries the precision with bit 4
    # set for 12-bit pixels
    import synth
    from paper_2207_05152_gb300 import model as M
    blob = M.fp32_blob12(synth.predictive_mlp([12, 32, 32, 4096], 3, sigma=96.0, levels=4096))
    img = synth.phantom_image12(9, 14, 2)
    data = orc.encode(blob, img, 3)
    h = lib.dlic_read_header(data)
    assert (h["height"], h["width"], h["streams"], h["precision"]) == (9, 14, 3, 0x10)
    assert h["hash"] == orc.fnv1a64(blob)
    with pytest.raises(lib.DlicError) as e:
        lib.dlic_read_header(b"DLC2" + data[4:])
    assert e.value.code == lib.DLIC_ERR_CORRUPT


def test_trainer_modes_are_checked_before_any_device_call(lib):
    # DLIC_TRAIN_RECOMPUTE takes a BF16 mode; unknown modes are refused; the
    # checks run before the trainer allocates anything (no GPU here)
    params = np.zeros(lib.dlic_train_param_count(12, 32, 32), np.float32)
    for mode in (lib.DLIC_TRAIN_FP32 | lib.DLIC_TRAIN_RECOMPUTE, 7, 7 | lib.DLIC_TRAIN_RECOMPUTE):
        with pytest.raises(Exception) as e:
            lib.dlic_trainer_create_k(12, 32, 32, 256, mode, 256, params)
        assert "mode" in str(e.value).lower() or "recompute" in str(e.value).lower()
