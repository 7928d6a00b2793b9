"""Multi-process paths on CPU with the gloo backend, world size 2: the bench's timing reductions and
event sharding, and a seed-range split of one turn partition whose merged selection must equal the
unsharded oracle's (Sec. 2.1 selection order: lowest RSS, ties by lowest seed index)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1911_09340_gb300 import multi


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _bench_reductions(rank, world, port, out):
    dist = _init(rank, world, port)
    import bench
    t = bench.max_over_ranks(1.5 + rank, world)
    s = bench.sum_over_ranks(10.0 * (rank + 1), world)
    bench.barrier(world)
    out[rank] = (t, s, multi.event_indices(3, rank, world))
    dist.destroy_process_group()


def _seed_shards(rank, world, port, out):
    dist = _init(rank, world, port)
    import oracle as O
    from paper_1911_09340_gb300 import synth
    ev = synth.make_event_fixed(synth.make_chamber(), np.random.default_rng(3), counts=(3, 3, 4, 4))
    seeds = O.lattice(ev.partitions[0])
    b, e = multi.shard_range(seeds.shape[0], rank, world)
    P = O.Params(n_steps=ev.n_steps[0])
    r = O.scan(synth.uniform_field(1.0), P, seeds[b:e], -1, O.wires_aos(ev.wires), ev.hit_offsets,
               ev.drift, np.zeros(ev.n_hits, np.uint8), nthreads=2)
    li, lv = O.select(r["rss"], 5)
    idx, vals = multi.allgather_topk(lv, li + b, 5)
    out[rank] = (idx, vals)
    dist.destroy_process_group()


def _run(fn):
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(fn, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    return dict(out)


def test_bench_reductions_and_event_sharding_gloo():
    out = _run(_bench_reductions)
    for rank in (0, 1):
        t, s, ev = out[rank]
        assert t == 2.5 and s == 30.0
    assert out[0][2] == [0, 2, 4] and out[1][2] == [1, 3, 5]


def test_seed_sharded_selection_equals_unsharded_gloo():
    import oracle as O
    from paper_1911_09340_gb300 import synth
    out = _run(_seed_shards)
    ev = synth.make_event_fixed(synth.make_chamber(), np.random.default_rng(3), counts=(3, 3, 4, 4))
    seeds = O.lattice(ev.partitions[0])
    r = O.scan(synth.uniform_field(1.0), O.Params(n_steps=ev.n_steps[0]), seeds, -1,
               O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, np.zeros(ev.n_hits, np.uint8))
    ri, rv = O.select(r["rss"], 5)
    for rank in (0, 1):
        idx, vals = out[rank]
        assert idx == list(ri) and np.array_equal(vals, rv)


def test_shard_range_and_merge_rules():
    for total in (0, 1, 7, 144):
        for world in (1, 2, 3, 8):
            spans = [multi.shard_range(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(e - b for b, e in spans) - min(e - b for b, e in spans) <= 1
    idx, vals = multi.merge_topk([[0.5, float("nan")], [0.5, 0.25]], [[7, 1], [3, 9]], 4)
    assert idx == [9, 3, 7, 1]
