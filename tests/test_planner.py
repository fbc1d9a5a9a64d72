"""The wavefront decoder's shared-memory planner (host code in decode_tc.cu),
compiled with nvcc into a host program and run on the CPU: which prior store
each case gets, and that every accepted plan fits the shared memory."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
LIMIT = 232448 - 5120


@pytest.fixture(scope="module")
def plans():
    if not (os.path.exists(NVCC) or shutil.which("nvcc")):
        pytest.skip("nvcc is not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "planner_check")
        cmd = [NVCC if os.path.exists(NVCC) else "nvcc", "-std=c++17", "--expt-relaxed-constexpr",
               "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(HERE, "..", "include"),
               "-o", exe, os.path.join(HERE, "planner_check.cu")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    res = {}
    for line in out.splitlines():
        name, *v = line.split()
        if name == "clusters":
            res["clusters_" + v[0]] = [int(x) for x in v[1:]]
            continue
        if name == "deep":
            ok, deep, nhh, smma, nt, gimg, total = map(int, v[1:])
            res["deep_" + v[0]] = dict(ok=ok, deep=deep, nhh=nhh, smma=smma, nt=nt, gimg=gimg, total=total)
            continue
        ok, nt, tq, gimg, ring_rows, list_rows, lut2, total = map(int, v)
        res[name] = dict(ok=ok, nt=nt, tq=tq, gimg=gimg, ring_rows=ring_rows, list_rows=list_rows, lut2=lut2,
                         total=total)
    return res


def test_accepted_plans_fit(plans):
    for name, p in plans.items():
        if isinstance(p, dict) and p["ok"]:
            assert 0 < p["total"] <= LIMIT, name


def test_default_image_gets_the_tagged_ring(plans):
    p = plans["int8_default_512"]
    assert p["ok"] and p["tq"] > 0 and p["gimg"] == 0 and p["lut2"] == 1 and p["nt"] == 16


def test_forced_plans(plans):
    assert plans["int8_byte_ring_512"]["tq"] == 0 and plans["int8_byte_ring_512"]["gimg"] == 0
    assert plans["int8_image_512"]["gimg"] == 1 and plans["int8_image_512"]["ring_rows"] == 0


def test_big_fp32_window_drops_the_tagged_ring(plans):
    # 78 inputs x 128 units of FP32 weights leave no room for the tagged ring
    p = plans["fp32_fig6_512"]
    assert p["ok"] and p["tq"] == 0 and p["gimg"] == 0


def test_long_waves_read_the_image_and_longer_ones_are_refused(plans):
    assert plans["int8_wide_4096x12288"]["ok"] and plans["int8_wide_4096x12288"]["gimg"] == 1
    assert not plans["int8_huge_30000x90000"]["ok"]


def test_volumes(plans):
    p = plans["int8_volume_35x256"]
    assert p["ok"] and p["gimg"] == 1 and p["tq"] == 0
    # 35 slices can be active at once, each with ceil(86 / 16) rows of a CTA
    assert p["list_rows"] >= 35 * 6
    assert plans["grid_volume_128x512"]["ok"] and plans["grid_batch_64x1536x2048"]["ok"]


def test_autotuner_cluster_sizes(plans):
    # one image gets the largest cluster; a batch shares the SMs (power-of-two
    # clusters of at most 16, at most one CTA per SM in all); tiny images that
    # already fill the GPU keep one CTA each
    assert plans["clusters_single_512"] == [16]
    ps = plans["clusters_batch64"]
    assert all(p in (1, 2, 4, 8, 16) for p in ps) and sum(ps) <= 152 and max(ps) > 1
    assert plans["clusters_tiny200"] == [1, 1]


def test_deeper_networks_take_the_warp_mma_chain(plans):
    # six dense layers (four hidden-to-hidden layers of 128 units in shared
    # memory) and a single hidden layer: warp-level MMAs on chunks of at most
    # 32 pixels, every plan within the shared memory, the long waves of a
    # 4096 x 12288 image reading their priors back from the image
    for name in ("six_layers_512", "six_layers_512_one_cta", "one_hidden_512", "six_layers_4096x12288"):
        p = plans["deep_" + name]
        assert p["ok"] and p["deep"] == 1 and p["smma"] == 1 and 16 <= p["nt"] <= 32, name
        assert 0 < p["total"] <= LIMIT, name
    assert plans["deep_six_layers_512"]["nhh"] == 4 and plans["deep_one_hidden_512"]["nhh"] == 0
    assert plans["deep_six_layers_512"]["gimg"] == 0 and plans["deep_six_layers_4096x12288"]["gimg"] == 1
