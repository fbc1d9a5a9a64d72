"""dlic_encode_noalloc: the encoder for callers that cannot allocate device
memory (for example a plug-in inside a framework that owns every device
allocation).  It must produce exactly the bitstreams of dlic_encode, call
after call, although every call reuses the library's one fixed scratch block
with whatever the previous call left in it.

Named to be collected last, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest
import torch

import synth
from paper_2207_05152_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2207_05152_gb300 import _lib
    return _lib


def _encode_both(lib, codec, img, streams):
    t = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    desc = codec._desc([t])
    cap = codec.capacity([img.shape], [streams])
    # reference: the existing entry point with a caller-provided workspace
    ref, ref_offs = codec.encode([t], [streams])
    # the no-allocation entry point; output buffers still come from the caller
    out = torch.full((cap,), 0xA5, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(2, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lib.dlic_encode_noalloc(codec.handle, desc, [streams], out.data_ptr(), out.numel(), offs.data_ptr(),
                            status.data_ptr(), stream)
    torch.cuda.synchronize()
    n_ref = int(ref_offs[1].item())
    n_new = int(offs[1].item())
    assert int(status.item()) == 0
    assert n_new == n_ref
    assert torch.equal(out[:n_new], ref[:n_ref])
    return out[:n_new].cpu().numpy().tobytes()


def test_noalloc_matches_dlic_encode_twice(lib):
    from paper_2207_05152_gb300.codec import Codec
    _, blob8, _ = workloads.models()
    codec = Codec(blob8)
    first = workloads.cfg2_image()
    second = synth.voronoi_image(300, 700, 77)
    a = _encode_both(lib, codec, first, 256)
    b = _encode_both(lib, codec, second, 64)    # the block still holds the first call's data
    assert a != b
    dec, st = codec.decode_bytes([a, b])
    assert st == [0, 0]
    assert np.array_equal(dec[0], first) and np.array_equal(dec[1], second)
    codec.close()


def test_noalloc_rejects_batches_beyond_its_block(lib):
    from paper_2207_05152_gb300.codec import Codec
    _, blob8, _ = workloads.models()
    codec = Codec(blob8)
    big = torch.zeros((2048, 2048), dtype=torch.uint8, device="cuda")   # needs ~25 MB of scratch
    out = torch.empty(codec.capacity([(2048, 2048)]), dtype=torch.uint8, device="cuda")
    offs = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(lib.DlicError) as e:
        lib.dlic_encode_noalloc(codec.handle, codec._desc([big]), None, out.data_ptr(), out.numel(),
                                offs.data_ptr(), 0, 0)
    assert e.value.code == lib.DLIC_ERR_CAPACITY
    assert "scratch" in str(e.value)
    codec.close()
