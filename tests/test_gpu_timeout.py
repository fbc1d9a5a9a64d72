"""Bounded waits of the wavefront decoders: a wait on another CTA that runs
out ends the call with DLIC_ERR_TIMEOUT and leaves the device usable.

The decoders wait for other CTAs in two places: a pixel that a neighbouring
CTA of the cluster pushes into the tagged ring, and the grid-wide barrier
between waves (DLIC_PLAN_GRID).  With the peer wait limit set to a few
hundred cycles both waits run out on every call: on the ring, the CTA that
owns row 1 reaches wave 3 after three empty waves and then waits for the
pixels row 0's CTA decodes in waves 0..2 (each a chain of thousands of
cycles); at the grid barrier after wave 0, the CTAs without a pixel wait for
the one CTA that decodes pixel (0, 0).  Afterwards the default limit is
restored and the same call must decode the image exactly."""
import numpy as np
import pytest
import torch

from paper_2207_05152_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300 import _lib
    return _lib


@pytest.mark.parametrize("prec,plan", [("int8", "auto"), ("fp32", "auto"), ("int8", "grid"), ("fp32", "grid")])
def test_peer_wait_that_runs_out_reports_timeout(lib, prec, plan):
    from paper_2207_05152_gb300.codec import Codec
    _, blob8, blob32 = workloads.models()
    blob = blob8 if prec == "int8" else blob32
    code = {"auto": lib.DLIC_PLAN_AUTO, "grid": lib.DLIC_PLAN_GRID}[plan]
    img = workloads.cfg2_image()
    codec = Codec(blob, decode_plan=code)
    bits = codec.encode_to_bytes([torch.from_numpy(img).cuda()], [256])
    lib.dlic_model_set_peer_wait_limit(codec.handle, 300)
    for _ in range(2):
        _, st = codec.decode_bytes(bits)
        assert st == [lib.DLIC_ERR_TIMEOUT]
    lib.dlic_model_set_peer_wait_limit(codec.handle, 0)   # back to the default
    dec, st = codec.decode_bytes(bits)
    assert st == [0] and np.array_equal(dec[0], img)
    codec.close()
