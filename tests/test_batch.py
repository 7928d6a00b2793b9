"""Batches of events (comet_scan_batch): the batched launches compute exactly what the per-event
calls compute (same kernels' arithmetic, same inputs), so every partition's best seed, its RSS and
the hit classes must be identical to the per-event scan, with and without the CUDA graph, with slots
refilled as events finish and with a seed budget that makes slots wait."""
import numpy as np
import pytest

from paper_1911_09340_gb300 import synth

pytestmark = pytest.mark.gpu


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
    best, table = batch.autotune(bs, events[:3], slots_options=(2, 4), ctas_options=(0, 2),
                                 graph_options=(True, False))
    assert len(table) == 8 and best in table
    r = bs.run(events, collect=True)
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
