"""Batches of events (comet_scan_batch): the batched launches compute exactly what the per-event
calls compute (same kernels' arithmetic, same inputs), so every partition's best seed, its RSS and
the hit classes must be identical to the per-event scan, with and without the CUDA graph, with slots
refilled as events finish and with a seed budget that makes slots wait."""
import numpy as np
import pytest

from paper_1911_09340_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _one_warp_per_32_seeds(ctx):
    """The batched launches record one warp per 32 seeds; the per-event reference records the same
    way here (comet_ctx_set_record_blocks(0)), so that the two agree bit for bit in FP64 too."""
    ctx.set_record_blocks(0)
    yield
    ctx.set_record_blocks(1)


def _events(n):
    return [synth.batch_event(i, counts_scale=3) for i in range(n)]


def _reference(ctx, events, dtype, stride):
    import torch
    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import scan
    field = B.DeviceField.from_synth(synth.uniform_field(1.0))
    S = max(sp.n_seeds for ev in events for sp in ev.partitions)
    n_rec = max(n // stride + 1 for ev in events for n in ev.n_steps)
    H = max(ev.n_hits for ev in events)
    ws = scan.Workspace(S, n_rec, H, dtype)
    out = []
    for ev in events:
        dev = scan.DeviceEvent.from_event(ev, dtype)
        out.append(scan.scan_event(ctx, field, ev, dev, ws, dtype, stride, 1e-2, collect=True))
    return out


@pytest.mark.parametrize("dtype_name,graph,budget", [("float32", True, 1 << 20), ("float64", False, 1 << 20),
                                                      ("float32", True, 6000)])
def test_batch_equals_per_event_scan(ctx, dtype_name, graph, budget):
    import torch
    from paper_1911_09340_gb300 import batch
    dtype = getattr(torch, dtype_name)
    events = _events(9)
    ref = _reference(ctx, events, dtype, 16)
    bs = batch.BatchScanner(ctx, dtype, stride=16, lam=1e-2, slots=4, max_seeds=4096,
                            max_total_seeds=budget, max_wires=512, max_hits=1024, graph=graph)
    r = bs.run(events, collect=True)
    for ev, rr, res in zip(events, ref, r["results"]):
        assert len(res.best_idx) == len(ev.partitions)
        for p, part in enumerate(rr):
            assert res.best_idx[p] == part["idx"]
            assert res.best_rss[p] == part["rss"]
            assert np.array_equal(res.hit_class[p], part["hit_class"])
    assert np.all(r["latency_ms"] > 0) and r["rounds"] >= max(len(ev.partitions) for ev in events)


@pytest.mark.parametrize("dtype_name,solo_lanes", [("float32", 1), ("float32", 3), ("float64", 2)])
def test_size_aware_rounds_equal_per_event_scan(ctx, dtype_name, solo_lanes):
    """Partitions of at least 256 seeds run through the single-event calls on 1-3 solo lanes (each
    with its own context and stream) while the smaller ones are batched: every partition's results
    are still identical to the per-event scan."""
    import torch
    from paper_1911_09340_gb300 import batch
    dtype = getattr(torch, dtype_name)
    events = _events(9)
    sizes = {sp.n_seeds for ev in events for sp in ev.partitions}
    assert min(sizes) < 256 <= max(sizes)          # both kinds of partition occur
    ref = _reference(ctx, events, dtype, 16)
    bs = batch.BatchScanner(ctx, dtype, stride=16, lam=1e-2, slots=4, max_seeds=4096,
                            max_total_seeds=1 << 16, max_wires=512, max_hits=1024, graph=True,
                            solo_min_seeds=256, solo_lanes=solo_lanes)
    try:
        r = bs.run(events, collect=True)
        for ev, rr, res in zip(events, ref, r["results"]):
            assert len(res.best_idx) == len(ev.partitions)
            for p, part in enumerate(rr):
                assert res.best_idx[p] == part["idx"] and res.best_rss[p] == part["rss"]
                assert np.array_equal(res.hit_class[p], part["hit_class"])
    finally:
        bs.close_lanes()


@pytest.mark.parametrize("chunk_wires,item_groups", [(8, 2), (64, 0), (0, 5)])
def test_chunk_and_item_knobs_equal_per_event_scan(ctx, chunk_wires, item_groups):
    """The DCA's wires per chunk (a context setting, shared by both paths) and the batched DCA's
    seed groups per item: batched results stay bit-identical to the per-event scan of the same
    context setting."""
    import torch
    from paper_1911_09340_gb300 import batch
    events = _events(6)
    ctx.set_dca_chunk_wires(chunk_wires)
    try:
        ref = _reference(ctx, events, torch.float32, 16)
        bs = batch.BatchScanner(ctx, torch.float32, stride=16, lam=1e-2, slots=3, max_seeds=4096,
                                max_total_seeds=1 << 15, max_wires=512, max_hits=1024,
                                chunk_wires=chunk_wires, item_groups=item_groups)
        r = bs.run(events, collect=True)
        for ev, rr, res in zip(events, ref, r["results"]):
            for p, part in enumerate(rr):
                assert res.best_idx[p] == part["idx"] and res.best_rss[p] == part["rss"]
                assert np.array_equal(res.hit_class[p], part["hit_class"])
    finally:
        ctx.set_dca_chunk_wires(0)


def test_autotune_then_run_matches_per_event_scan(ctx):
    """The autotuner cycles through configurations (new caps reallocate the context's staging, and
    graphs captured before must be dropped); the configured run afterwards still reproduces the
    per-event scan exactly."""
    import torch
    from paper_1911_09340_gb300 import batch
    events = _events(6)
    ref = _reference(ctx, events, torch.float32, 16)
    bs = batch.BatchScanner(ctx, torch.float32, stride=16, lam=1e-2, slots=4, max_seeds=4096,
                            max_total_seeds=1 << 16, max_wires=512, max_hits=1024)
    try:
        best, table = batch.autotune(bs, events[:3], slots_options=(2, 4), ctas_options=(0, 2),
                                     graph_options=(True, False), chunk_options=(0, 16),
                                     item_options=(0, 8))
        assert len(table) == 11 and best in table
        # the per-event reference with the chunk width the autotuner left on the context
        ref = _reference(ctx, events, torch.float32, 16)
        r = bs.run(events, collect=True)
    finally:
        ctx.set_dca_chunk_wires(0)
    for rr, res in zip(ref, r["results"]):
        for p, part in enumerate(rr):
            assert res.best_idx[p] == part["idx"] and res.best_rss[p] == part["rss"]
            assert np.array_equal(res.hit_class[p], part["hit_class"])


def test_two_interleaved_scanners_match_per_event_scan(ctx):
    """Two scanners, each with its own context and stream, take alternate events and launch their
    rounds alternately: every event's results are still those of the per-event scan."""
    import torch
    from paper_1911_09340_gb300 import batch
    from paper_1911_09340_gb300 import binding as B
    events = _events(7)
    ref = _reference(ctx, events, torch.float32, 16)
    ctx2 = B.Context(torch.cuda.current_device())
    try:
        pair = [batch.BatchScanner(c, torch.float32, stride=16, lam=1e-2, slots=3, max_seeds=4096,
                                   max_total_seeds=1 << 15, max_wires=512, max_hits=1024, graph=g)
                for c, g in ((ctx, True), (ctx2, False))]
        r = batch.run_interleaved(pair, events, collect=True)
        for ev, rr, res in zip(events, ref, r["results"]):
            assert len(res.best_idx) == len(ev.partitions)
            for p, part in enumerate(rr):
                assert res.best_idx[p] == part["idx"] and res.best_rss[p] == part["rss"]
                assert np.array_equal(res.hit_class[p], part["hit_class"])
        assert np.all(r["latency_ms"] > 0)
        del pair
        torch.cuda.synchronize()
    finally:
        ctx2.close()


def _variant(ev, keep=None, extra_wires=0, seed=0):
    """An event with only the wires ``keep`` (indices into ev's wires), or with ``extra_wires``
    random chamber wires added, each with one noise hit (drift ~ U(0, 8 mm)); CSR order kept."""
    import dataclasses
    ch = synth.make_chamber()
    rng = np.random.default_rng(seed)
    offs = np.asarray(ev.hit_offsets)
    ids = list(range(ev.n_wires)) if keep is None else list(keep)
    hits = [np.arange(offs[i], offs[i + 1]) for i in ids]
    wire_ids = [int(ev.wire_ids[i]) for i in ids]
    cols = [ev.wires[:, i] for i in ids]
    drift = [ev.drift[h] for h in hits]
    turn = [ev.hit_turn[h] for h in hits]
    dtrue = [ev.hit_dtrue[h] for h in hits]
    if extra_wires:
        new = rng.choice(np.setdiff1d(np.arange(ch.n_wires), ev.wire_ids), size=extra_wires, replace=False)
        for w in new:
            wire_ids.append(int(w))
            cols.append(np.concatenate([ch.a[:, w], ch.u[:, w]]))
            drift.append(rng.uniform(0, 8e-3, size=1))
            turn.append(np.array([-1], np.int32))
            dtrue.append(np.array([np.nan]))
    order = np.argsort(wire_ids, kind="stable")
    counts = np.array([len(drift[i]) for i in order])
    o = np.zeros(len(order) + 1, np.int32)
    o[1:] = np.cumsum(counts)
    return dataclasses.replace(
        ev, wire_ids=np.array(wire_ids, np.int32)[order], wires=np.stack([cols[i] for i in order], 1),
        hit_offsets=o, drift=np.concatenate([drift[i] for i in order]),
        hit_turn=np.concatenate([turn[i] for i in order]).astype(np.int32),
        hit_dtrue=np.concatenate([dtrue[i] for i in order]))


@pytest.mark.parametrize("dtype_name", ["float32", "float64"])
def test_batch_matches_oracle(ctx, dtype_name):
    """The batched path against the oracle, not only against the per-event path: events of 1-6 turns
    (small lattices), among them one reduced to a single wire (W = 1) and one with 300 extra wires
    (W > 256); every partition's selected seed by the argmin rule (identical, or oracle RSS within
    1e-5 relative of the oracle's minimum over all seeds), its RSS (FP64 within 1e-10 relative; FP32
    within the bound of the 2 um DCA bar), its hit classes bit-identical except within 1 um (FP32) /
    1e-9 m (FP64) of the cutoff, and the mask carried from partition to partition."""
    import torch

    import oracle as O
    from gpu_util import CLASS_EDGE, FP32_DCA_TOL, per_wire_residual, rss_bound, seen
    from paper_1911_09340_gb300 import batch
    dtype = getattr(torch, dtype_name)
    evs = [synth.batch_event(i, counts_scale=3) for i in range(12)]
    by_turns = {}
    for ev in evs:
        by_turns.setdefault(len(ev.partitions), ev)
    events = [by_turns[k] for k in sorted(by_turns)]
    events.append(_variant(events[0], keep=[int(np.argmax(np.diff(events[0].hit_offsets)))]))
    events.append(_variant(events[-2], extra_wires=300, seed=3))
    assert events[-2].n_wires == 1 and events[-1].n_wires > 256
    assert len({len(ev.partitions) for ev in events}) >= 4
    stride, lam = 32, 1e-2
    bs = batch.BatchScanner(ctx, dtype, stride=stride, lam=lam, slots=4, max_seeds=1 << 12,
                            max_total_seeds=1 << 14, max_wires=1024, max_hits=2048, graph=False)
    r = bs.run(events, collect=True)
    field = synth.uniform_field(1.0)
    for ev, res in zip(events, r["results"]):
        w, d = O.wires_aos(seen(ev.wires, dtype)), seen(ev.drift, dtype)
        wid = np.repeat(np.arange(ev.n_wires), np.diff(ev.hit_offsets))
        omask = np.zeros(ev.n_hits, np.uint8)
        assert len(res.best_idx) == len(ev.partitions)
        for p, spec in enumerate(ev.partitions):
            seeds = seen(O.lattice(spec), dtype)
            op = O.Params(n_steps=ev.n_steps[p], stride=stride, lam=lam, tol=1e-12)
            o = O.scan(field, op, seeds, spec.charge, w, ev.hit_offsets, d, omask)
            o_idx, o_best = O.select(o["rss"], 1)
            g = res.best_idx[p]
            assert g == int(o_idx[0]) or o["rss"][g] <= o_best[0] * (1 + 1e-5), (p, g, int(o_idx[0]))
            one = O.scan(field, op, seeds[g:g + 1], spec.charge, w, ev.hit_offsets, d, omask,
                         want_dca=True)
            if dtype == torch.float64:
                assert abs(res.best_rss[p] - one["rss"][0]) <= 1e-10 * one["rss"][0] + 1e-300
            else:
                e = per_wire_residual(one["dca"], ev.hit_offsets, d, omask)
                assert abs(res.best_rss[p] - one["rss"][0]) <= rss_bound(e, lam, FP32_DCA_TOL)[0] + 1e-12
            cls, dwr, m2 = O.classify(field, op, seeds[g], spec.charge, w, ev.hit_offsets, d, omask,
                                      update_mask=True)
            edge = np.abs(np.abs(dwr[wid] - d) - lam) < CLASS_EDGE[dtype]
            diff = np.flatnonzero(res.hit_class[p] != cls)
            assert np.all(edge[diff]), (p, diff[~edge[diff]])
            omask = np.maximum(omask, res.hit_class[p].astype(np.uint8))
            assert np.array_equal(omask[~edge], m2[~edge])
