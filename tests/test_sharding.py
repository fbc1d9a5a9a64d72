"""The multi-GPU split (paper_2207_05152_gb300/sharding.py) on CPU ranks.

Coding: the longest-processing-time partition of a batch by pixel count,
checked against brute force on small batches; with two gloo ranks each
encoding its own images (the oracle stands in for a GPU's encoder), the
all-gathered offsets lay the bitstreams out exactly as one process would.
Training: with two gloo ranks holding uneven halves of a batch, the weighted
all-reduce of their FP64 gradients (the oracle's) equals the gradient of the
whole batch, and every rank applies the same update."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2207_05152_gb300 import sharding  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(target, world, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    import queue
    import time
    res, t0 = [], time.time()
    while len(res) < world:
        try:
            res.append(q.get(timeout=2))
        except queue.Empty:
            # a rank that failed before reporting ends the test at once
            assert all(p.exitcode in (None, 0) for p in procs), [p.exitcode for p in procs]
            assert time.time() - t0 < 300, "ranks did not report"
    res.sort(key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def test_lpt_against_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(40):
        n, m = int(rng.integers(1, 8)), int(rng.integers(1, 4))
        px = [int(v) for v in rng.integers(1, 100, n)]
        owners, load = sharding.lpt_partition(px, m)
        assert sorted(set(owners)) <= list(range(m)) and len(owners) == n
        assert [sum(p for p, o in zip(px, owners) if o == r) for r in range(m)] == load
        best = min(max(sum(p for p, o in zip(px, a) if o == r) for r in range(m))
                   for a in itertools.product(range(m), repeat=n))
        # Graham's bound for the longest-processing-time rule
        assert max(load) <= (4.0 / 3.0 - 1.0 / (3.0 * m)) * best + 1e-9
    # deterministic, and one rank takes everything
    assert sharding.lpt_partition([5, 5, 3], 2) == ([0, 1, 0], [8, 5])
    assert sharding.lpt_partition([7, 1, 2], 1) == ([0, 0, 0], [10])
    with pytest.raises(ValueError):
        sharding.lpt_partition([1], 0)


def test_cfg4_batch_is_balanced():
    import synth
    sizes = [h * w for h, w in synth.uneven_sizes(64, 4000)]
    for m in (2, 4, 8):
        owners, load = sharding.lpt_partition(sizes, m)
        assert max(load) - min(load) <= max(sizes)
        assert max(load) <= 1.02 * sum(sizes) / m + max(sizes) / 3


def _coding_rank(rank, world, port, q, shapes):
    dist = _init(rank, world, port)
    import oracle
    import synth
    from paper_2207_05152_gb300 import model as M
    blob = M.fp32_blob(synth.predictive_mlp([12, 32, 32, 256], 4))
    imgs = [synth.voronoi_image(h, w, 60 + i) for i, (h, w) in enumerate(shapes)]
    owners, _ = sharding.lpt_partition([i.size for i in imgs], world)
    mine = sharding.shard_of(owners, rank)
    local = {i: oracle.encode(blob, imgs[i], 3) for i in mine}
    offs = sharding.gather_offsets([len(local[i]) for i in mine], owners, rank)
    everything = [None] * world
    dist.all_gather_object(everything, local)
    dist.destroy_process_group()
    q.put((rank, offs, mine, everything))


def test_sharded_coding_offsets_gloo():
    import oracle
    import synth
    from paper_2207_05152_gb300 import model as M
    shapes = [(9, 30), (20, 11), (5, 5), (14, 40), (3, 60), (12, 12), (30, 7)]
    res = _run_ranks(_coding_rank, 2, shapes)
    blob = M.fp32_blob(synth.predictive_mlp([12, 32, 32, 256], 4))
    want = [oracle.encode(blob, synth.voronoi_image(h, w, 60 + i), 3) for i, (h, w) in enumerate(shapes)]
    want_offs = np.concatenate([[0], np.cumsum([len(b) for b in want])]).tolist()
    shards = []
    for rank, offs, mine, everything in res:
        assert offs == want_offs                   # every rank has the whole layout
        shards.append(set(mine))
        merged = {k: v for part in everything for k, v in part.items()}
        for i, b in merged.items():
            assert b == want[i]
            assert offs[i + 1] - offs[i] == len(b)
    assert shards[0].isdisjoint(shards[1]) and shards[0] | shards[1] == set(range(len(shapes)))


def _training_rank(rank, world, port, q, split):
    dist = _init(rank, world, port)
    import torch
    import synth
    from oracle import train64
    from paper_2207_05152_gb300 import train as T
    imgs = [synth.config_image(3, i) for i in range(2)]
    ctx, tgt = T.sample_contexts(imgs, 1024, 21)
    layers = synth.xavier_mlp([12, 24, 24, 256], 22)
    lo, hi = (0, split) if rank == 0 else (split, 1024)

    def backward(c, t):
        g, loss = train64.gradient(layers, c, t)
        return loss, torch.from_numpy(np.concatenate([a.reshape(-1) for wb in g for a in wb]))

    applied = []
    loss = sharding.data_parallel_step(backward, applied.append, ctx[lo:hi], tgt[lo:hi])
    dist.destroy_process_group()
    q.put((rank, loss, applied[0].numpy()))


@pytest.mark.parametrize("split", [512, 700])
def test_data_parallel_gradient_equals_full_batch_gloo(split):
    import synth
    from oracle import train64
    from paper_2207_05152_gb300 import train as T
    res = _run_ranks(_training_rank, 2, split)
    imgs = [synth.config_image(3, i) for i in range(2)]
    ctx, tgt = T.sample_contexts(imgs, 1024, 21)
    layers = synth.xavier_mlp([12, 24, 24, 256], 22)
    g, loss = train64.gradient(layers, ctx, tgt)
    full = np.concatenate([a.reshape(-1) for wb in g for a in wb])
    for rank, l, applied in res:
        assert l == pytest.approx(loss, rel=1e-12)
        np.testing.assert_allclose(applied, full, rtol=1e-10, atol=1e-15)
    np.testing.assert_array_equal(res[0][2], res[1][2])   # the same update on every rank
