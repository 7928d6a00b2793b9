"""End-to-end parity of the partition pipeline (lattice -> propagate -> dca -> select -> classify ->
mask) run through the package's scan driver, against the oracle's pipeline.

Bars: the argmin seed identical, or its oracle RSS within 1e-5 relative of the oracle's minimum;
classifications bit-identical except hits whose residual lies within 1 um (FP32; 1e-9 m FP64) of
lambda.  The benchmark's launch configuration (2^18 seeds per partition, FP32, stride 32) is checked
against the oracle on every seed of every partition of three benchmark events; the other strides
and the 2^24-seed partition on samples of seeds the oracle computes one by one.  No statistical
allowance: every compared value must meet its bar.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1911_09340_gb300 import binding as B
from paper_1911_09340_gb300 import scan, synth

from gpu_util import CLASS_EDGE, FP32_DCA_TOL, per_wire_residual, rss_bound, seen

pytestmark = pytest.mark.gpu
UNIFORM = synth.uniform_field(1.0)


def test_single_event_fp64_all_partitions(ctx):
    ev = synth.single_event_fp64()
    f = B.DeviceField.from_synth(UNIFORM)
    dev = scan.DeviceEvent.from_event(ev, torch.float64)
    n_rec = max(ev.n_steps) + 1
    ws = scan.Workspace(ev.partitions[0].n_seeds, n_rec, ev.n_hits, torch.float64)
    omask = np.zeros(ev.n_hits, np.uint8)
    for part, (spec, bp) in enumerate(zip(ev.partitions, scan.event_params(ev, torch.float64))):
        scan.scan_partition(ctx, f, bp, spec, dev, ws)
        torch.cuda.synchronize()
        g_rss = ws.rss[:spec.n_seeds].cpu().numpy()
        g_idx = int(ws.idx[0])
        g_cls = ws.hit_class[:ev.n_hits].cpu().numpy()
        op = O.Params(n_steps=bp.n_steps, stride=bp.stride, lam=bp.lam, tol=1e-12)
        r = O.scan_partition(UNIFORM, op, spec, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, omask)
        assert np.allclose(g_rss, r["rss"], rtol=1e-10, atol=0)
        assert g_idx == int(r["idx"][0]) or r["rss"][g_idx] <= r["best_rss"][0] * (1 + 1e-5)
        assert np.array_equal(g_cls, r["hit_class"])
        assert np.array_equal(dev.mask[:ev.n_hits].cpu().numpy(), r["mask"])
        omask = r["mask"]


def _edge_hits(dca_wire, ev, drift, lam, band):
    """Hits whose residual |D - r| (D: the oracle's DCA of the classified seed to the hit's wire)
    lies within `band` of the cutoff: the only hits whose class may differ."""
    wid = np.repeat(np.arange(ev.n_wires), np.diff(ev.hit_offsets))
    return np.abs(np.abs(dca_wire[wid] - drift) - lam) < band


def _check_selected_and_classified(g_rss, g_idx, g_cls, r_rss_of, seeds, ev, op, w32, d32, mask):
    """The argmin rule and the classification rule for one partition.  ``r_rss_of(i)`` is the
    oracle's RSS of seed i; returns the oracle's mask after classifying the selected seed."""
    o_best_idx, o_best = r_rss_of(None)
    # argmin seed identical, or its oracle RSS within 1e-5 relative of the oracle's minimum
    assert g_idx == o_best_idx or r_rss_of(g_idx) <= o_best * (1 + 1e-5), (g_idx, o_best_idx)
    # classification of the selected seed: bit-identical except within 1 um of the cutoff
    cls, dwr, m2 = O.classify(UNIFORM, op, seeds[g_idx], -1, O.wires_aos(w32), ev.hit_offsets, d32,
                              mask, update_mask=True)
    edge = _edge_hits(dwr, ev, d32, op.lam, CLASS_EDGE[torch.float32])
    diff = np.flatnonzero(g_cls != cls)
    assert np.all(edge[diff]), ("hits classified differently away from the cutoff", diff[~edge[diff]])
    return m2, int(edge.sum()), diff.size


HEADLINE_EVENTS = (0, 1, 2)


@pytest.mark.parametrize("event", HEADLINE_EVENTS)
def test_benchmark_event_every_partition_full_oracle(ctx, event):
    """The benchmark's launch configuration -- 2^18 seeds per turn partition, FP32, every 32nd state
    recorded, uniform 1 T -- on every partition of a benchmark event, against the oracle run on all
    2^18 seeds of each partition (same FP32-rounded seeds, wires and drifts), the hit mask carried
    from each partition's classification to the next.

    Per partition, through the scan driver (lattice -> propagate -> dca -> select -> classify, the
    DCA on its pruned path as the benchmark runs it):
      - every seed's RSS within the bound the 2 um DCA bar implies term by term, n_in identical
        for every seed with no residual within 2 um of the cutoff;
      - the selected seed identical to the oracle's argmin, or its oracle RSS within 1e-5 relative
        of the oracle's minimum over the whole partition;
      - the selected seed's hit classes bit-identical to the oracle's except hits whose residual
        lies within 1 um of the cutoff, and the carried mask equal to the oracle's;
    and, on the exact path (every DCA requested), every (seed, wire with an unmasked hit) DCA that
    can give a residual below lambda within 2 um of the oracle's, the others beyond the wire's
    capture radius on both sides."""
    ev = synth.multi_turn_event(event)
    S = ev.partitions[0].n_seeds
    assert S == 1 << 18
    f = B.DeviceField.from_synth(UNIFORM)
    dev = scan.DeviceEvent.from_event(ev, torch.float32)
    params = scan.event_params(ev, torch.float32, stride=32)
    ws = scan.Workspace(S, max(p.n_rec for p in params), ev.n_hits, torch.float32)
    w32, d32 = seen(ev.wires, torch.float32), seen(ev.drift, torch.float32)
    omask = np.zeros(ev.n_hits, np.uint8)
    dca = torch.empty((ev.n_wires, S), dtype=torch.float32, device="cuda")
    for part, (spec, bp) in enumerate(zip(ev.partitions, params)):
        assert np.array_equal(dev.mask[:ev.n_hits].cpu().numpy(), omask)
        seeds = O.lattice(spec).astype(np.float32).astype(np.float64)
        op = O.Params(n_steps=bp.n_steps, stride=bp.stride, lam=bp.lam, tol=1e-12)
        r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(w32), ev.hit_offsets, d32, omask,
                   want_dca=True)
        e = per_wire_residual(r["dca"], ev.hit_offsets, d32, omask)
        live = np.isfinite(e[0])
        # exact path: every DCA of a wire that is in the sum
        seeds_dev, charge, pts, nv, _, _ = ws.views(S, bp.n_rec)
        B.comet_scan_lattice(ctx, spec, seeds_dev, charge)
        B.comet_scan_propagate(ctx, f, bp, seeds_dev, charge, pts, nv)
        rss_x = torch.empty(S, dtype=torch.float32, device="cuda")
        nin_x = torch.empty(S, dtype=torch.int32, device="cuda")
        B.comet_scan_dca(ctx, f, bp, pts, nv, charge, dev.wires, dev.hit_offsets, dev.drift,
                         dev.mask, rss_x, nin_x, dca_out=dca, n_wires=ev.n_wires)
        # every (seed, wire) whose DCA can give a residual below lambda -- the oracle's DCA within
        # the wire's capture radius (largest unmasked drift + lambda) plus 1 mm -- agrees to 2 um;
        # beyond it both sides lie beyond the capture radius (the wire adds lambda^2 either way:
        # far from the track the closest recorded state may be a track end, where the extrapolated
        # DCA depends on rounding)
        g_dca = dca.double().cpu().numpy()                     # [W][S]
        o_dca = r["dca"].T                                      # [W][S]
        cap = np.array([max((d32[j] for j in range(ev.hit_offsets[i], ev.hit_offsets[i + 1])
                             if not omask[j]), default=-1.0) for i in range(ev.n_wires)]) + bp.lam
        rel = live[:, None] & (o_dca < cap[:, None] + 1e-3)
        dd = np.abs(g_dca - o_dca)[rel]
        assert dd.max() <= FP32_DCA_TOL, dd.max()
        far = live[:, None] & ~rel
        margin = g_dca[far] - np.broadcast_to(cap[:, None], far.shape)[far]
        assert margin.min() >= 0.0, (margin.min(), int((margin < 0).sum()))
        # pruned path, the benchmark's sequence
        scan.scan_partition(ctx, f, bp, spec, dev, ws)
        torch.cuda.synchronize()
        g_rss = ws.rss[:S].double().cpu().numpy()
        g_idx = int(ws.idx[0])
        g_cls = ws.hit_class[:ev.n_hits].cpu().numpy()
        assert g_rss[g_idx] == g_rss.min() and g_idx == int(np.flatnonzero(g_rss == g_rss.min())[0])
        bound = rss_bound(e, bp.lam, FP32_DCA_TOL)
        excess = np.abs(g_rss - r["rss"]) - bound
        assert excess.max() <= 1e-12, (int((excess > 1e-12).sum()), int(np.argmax(excess)))
        edge_s = (np.abs(e - bp.lam) < FP32_DCA_TOL).any(1)
        assert np.array_equal(ws.n_in[:S].cpu().numpy()[~edge_s], r["n_in"][~edge_s])
        o_idx, o_best = O.select(r["rss"], 1)
        rss_of = lambda i: (int(o_idx[0]), float(o_best[0])) if i is None else float(r["rss"][i])
        omask, n_edge, n_diff = _check_selected_and_classified(g_rss, g_idx, g_cls, rss_of, seeds, ev,
                                                               op, w32, d32, omask)
        print(f"event {event} partition {part}: {live.sum()} wires in the sum, {dd.size} (seed, "
              f"wire) DCAs within reach, max |dDCA| {dd.max():.2e} m, selected {g_idx} (oracle "
              f"{int(o_idx[0])}), {n_edge} hits within 1 um of the cutoff, {n_diff} hit classes "
              f"differ")
    assert np.array_equal(dev.mask[:ev.n_hits].cpu().numpy(), omask)


@pytest.mark.parametrize("stride", [1, 4, 16, 24])
def test_multi_turn_event_fp32_full_size_sampled(ctx, stride):
    """2^18 seeds at the other pinned strides: a sample of seeds (random, the 64 of lowest GPU RSS and
    the selected one) computed by the oracle one by one; every sampled RSS within the bound of the
    2 um DCA bar, the selected seed at least as good (by the oracle) as every sampled seed, and the
    selected seed's classification bit-identical except within 1 um of the cutoff."""
    ev = synth.multi_turn_event(4)
    spec = ev.partitions[0]
    S = spec.n_seeds
    assert S == 1 << 18
    f = B.DeviceField.from_synth(UNIFORM)
    dev = scan.DeviceEvent.from_event(ev, torch.float32)
    bp = scan.event_params(ev, torch.float32, stride=stride)[0]
    ws = scan.Workspace(S, bp.n_rec, ev.n_hits, torch.float32)
    scan.scan_partition(ctx, f, bp, spec, dev, ws)
    torch.cuda.synchronize()
    g_rss = ws.rss[:S].double().cpu().numpy()
    g_idx = int(ws.idx[0])
    assert g_rss[g_idx] == g_rss.min() and g_idx == int(np.flatnonzero(g_rss == g_rss.min())[0])
    g_cls = ws.hit_class[:ev.n_hits].cpu().numpy()
    w32, d32 = seen(ev.wires, torch.float32), seen(ev.drift, torch.float32)
    seeds = O.lattice(spec).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(0)
    order = np.argsort(g_rss, kind="stable")
    sample = np.unique(np.concatenate([rng.choice(S, 384, replace=False), order[:64], [g_idx]]))
    op = O.Params(n_steps=bp.n_steps, stride=bp.stride, lam=bp.lam, tol=1e-12)
    mask = np.zeros(ev.n_hits, np.uint8)
    r = O.scan(UNIFORM, op, seeds[sample], -1, O.wires_aos(w32), ev.hit_offsets, d32, mask,
               want_dca=True)
    e = per_wire_residual(r["dca"], ev.hit_offsets, d32, mask)
    bound = rss_bound(e, bp.lam, FP32_DCA_TOL)
    excess = np.abs(g_rss[sample] - r["rss"]) - bound
    assert excess.max() <= 1e-12, (int((excess > 1e-12).sum()), sample[int(np.argmax(excess))])
    r_best = r["rss"][np.searchsorted(sample, g_idx)]
    assert r_best <= r["rss"].min() * (1 + 1e-5)
    rss_of = lambda i: (g_idx, r_best) if i is None else r_best
    _check_selected_and_classified(g_rss, g_idx, g_cls, rss_of, seeds, ev, op, w32, d32, mask)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_pipelined_scanner_equals_partition_by_partition(ctx, dtype):
    """PipelinedScanner (the next partition's recording on a second stream beside the current
    partition's DCA, two workspaces) gives bit-identical RSS, best seeds, hit classes and masks to
    scan_partition one partition at a time, over several events back to back."""
    evs = [synth.multi_turn_event(i, counts=(8, 8, 16, 16)) for i in range(3)]
    f = B.DeviceField.from_synth(UNIFORM)
    S = evs[0].partitions[0].n_seeds
    n_rec = max(bp.n_rec for ev in evs for bp in scan.event_params(ev, dtype, stride=32))
    H = max(ev.n_hits for ev in evs)
    ref = []
    ws = scan.Workspace(S, n_rec, H, dtype)
    for ev in evs:
        dev = scan.DeviceEvent.from_event(ev, dtype)
        out = []
        for spec, bp in zip(ev.partitions, scan.event_params(ev, dtype, stride=32)):
            scan.scan_partition(ctx, f, bp, spec, dev, ws)
            out.append((ws.rss[:S].cpu().numpy().copy(), int(ws.idx[0]),
                        ws.hit_class[:ev.n_hits].cpu().numpy().copy()))
        ref.append((out, dev.mask[:ev.n_hits].cpu().numpy().copy()))
    pipe = scan.PipelinedScanner(ctx, f, S, n_rec, H, dtype)
    try:
        devs = [scan.DeviceEvent.from_event(ev, dtype) for ev in evs]
        got = []
        for ev, dev in zip(evs, devs):
            cls = torch.zeros((len(ev.partitions), max(ev.n_hits, 1)), dtype=torch.uint8, device="cuda")
            rs = []
            for p, (spec, bp) in enumerate(zip(ev.partitions, scan.event_params(ev, dtype, stride=32))):
                w = pipe.partition(bp, spec, dev, hit_class=cls[p])
                rs.append((w.rss[:S].clone(), w.idx[:1].clone()))
            got.append((rs, cls))
        torch.cuda.synchronize()
        for (out, mask), (rs, cls), ev, dev in zip(ref, got, evs, devs):
            for p, ((rss, idx, hc), (g_rss, g_idx)) in enumerate(zip(out, rs)):
                assert np.array_equal(g_rss.cpu().numpy(), rss)
                assert int(g_idx[0]) == idx
                assert np.array_equal(cls[p, :ev.n_hits].cpu().numpy(), hc)
            assert np.array_equal(dev.mask[:ev.n_hits].cpu().numpy(), mask)
    finally:
        pipe.close()


def test_backward_partition_fp64_matches_oracle(ctx):
    """The exit-side (backward) scan of turn partition 0 — flipped charge and momentum — through the
    library against the oracle's pipeline, same bars as the forward scan."""
    ev = synth.single_event_fp64()
    f = B.DeviceField.from_synth(UNIFORM)
    dev = scan.DeviceEvent.from_event(ev, torch.float64)
    spec = synth.backward_partition(ev, 0)
    bp = scan.params_for(spec, ev.n_steps[0], torch.float64)
    ws = scan.Workspace(spec.n_seeds, bp.n_rec, ev.n_hits, torch.float64)
    scan.scan_partition(ctx, f, bp, spec, dev, ws)
    torch.cuda.synchronize()
    op = O.Params(n_steps=bp.n_steps, stride=bp.stride, lam=bp.lam, tol=1e-12)
    r = O.scan_partition(UNIFORM, op, spec, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift,
                         np.zeros(ev.n_hits, np.uint8))
    g_rss = ws.rss[:spec.n_seeds].cpu().numpy()
    g_idx = int(ws.idx[0])
    assert np.allclose(g_rss, r["rss"], rtol=1e-10, atol=0)
    assert g_idx == int(r["idx"][0]) or r["rss"][g_idx] <= r["best_rss"][0] * (1 + 1e-5)
    assert np.array_equal(ws.hit_class[:ev.n_hits].cpu().numpy(), r["hit_class"])
    # the backward scan represents turn 0 and finds most of its hits, as the forward scan does
    from paper_1911_09340_gb300 import metrics as M
    m = M.stage_metrics(r["hit_class"].astype(bool), ev.hit_turn)
    rf = O.scan_partition(UNIFORM, op, ev.partitions[0], O.wires_aos(ev.wires), ev.hit_offsets,
                          ev.drift, np.zeros(ev.n_hits, np.uint8))
    mf = M.stage_metrics(rf["hit_class"].astype(bool), ev.hit_turn)
    assert m.turn == mf.turn == 0 and m.efficiency > 0.8
    assert abs(m.efficiency - mf.efficiency) <= 0.05


def test_stage_metrics_from_gpu_equal_oracle_at_0_8_mm(ctx):
    """Stage metrics (lambda = 0.8 mm, the paper's optimum) from the library's stages equal those
    from the oracle's stages, FP64, every partition of the single event."""
    from paper_1911_09340_gb300 import experiments as X
    from paper_1911_09340_gb300 import metrics as M
    ev = synth.single_event_fp64()
    f = B.DeviceField.from_synth(UNIFORM)
    dev = scan.DeviceEvent.from_event(ev, torch.float64)
    ws = scan.Workspace(ev.partitions[0].n_seeds, max(ev.n_steps) + 1, ev.n_hits, torch.float64)
    g = X.scan_stages(ctx, f, ev, dev, ws, ev.partitions, ev.n_steps, torch.float64, 1, 8e-4)
    omask = np.zeros(ev.n_hits, np.uint8)
    o = []
    for spec, n in zip(ev.partitions, ev.n_steps):
        r = O.scan_partition(UNIFORM, O.Params(n_steps=n, stride=1, lam=8e-4, tol=1e-12), spec,
                             O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, omask)
        o.append(r["hit_class"].astype(bool))
        omask = r["mask"]
    for a, b in zip(g, o):
        assert np.array_equal(a, b)
    assert M.event_metrics(g, ev.hit_turn) == M.event_metrics(o, ev.hit_turn)


def test_sixteen_million_seed_partition_needs_64bit_offsets(ctx):
    """2^24 seeds (a 64^4 lattice) at stride 32: the track points hold 6 x 70 x 2^24 = 7.0e9 values
    (28 GB), so offsets into them, into the search bounds and into the partial sums exceed 32 bits.
    Sampled seeds -- among them the last one, at the highest offsets -- and the selected seed
    against the oracle within the bound the FP32 DCAs imply; the selection is the argmin of the
    RSS the GPU computed."""
    ev = synth.multi_turn_event(4, counts=(64, 64, 64, 64))
    spec = ev.partitions[0]
    S = spec.n_seeds
    assert S == 1 << 24
    f = B.DeviceField.from_synth(UNIFORM)
    dev = scan.DeviceEvent.from_event(ev, torch.float32)
    bp = scan.event_params(ev, torch.float32, stride=32)[0]
    assert 6 * bp.n_rec * S > 1 << 32
    ws = scan.Workspace(S, bp.n_rec, ev.n_hits, torch.float32)
    scan.scan_partition(ctx, f, bp, spec, dev, ws)
    torch.cuda.synchronize()
    g_rss = ws.rss[:S].double().cpu().numpy()
    g_idx = int(ws.idx[0])
    assert g_rss[g_idx] == g_rss.min() and g_idx == int(np.flatnonzero(g_rss == g_rss.min())[0])
    assert np.all(g_rss >= 0) and np.all(np.isfinite(g_rss))
    del ws
    torch.cuda.empty_cache()
    seeds = O.lattice(spec).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(1)
    sample = np.unique(np.concatenate([rng.choice(S, 256, replace=False), [g_idx, S - 1, S - 33]]))
    op = O.Params(n_steps=bp.n_steps, stride=bp.stride, lam=bp.lam, tol=1e-12)
    mask = np.zeros(ev.n_hits, np.uint8)
    w32, d32 = seen(ev.wires, torch.float32), seen(ev.drift, torch.float32)
    r = O.scan(UNIFORM, op, seeds[sample], -1, O.wires_aos(w32), ev.hit_offsets, d32, mask,
               want_dca=True)
    e = per_wire_residual(r["dca"], ev.hit_offsets, d32, mask)
    bound = rss_bound(e, bp.lam, FP32_DCA_TOL)
    excess = np.abs(g_rss[sample] - r["rss"]) - bound
    assert excess.max() <= 1e-12, (int((excess > 1e-12).sum()), sample[int(np.argmax(excess))])
    r_best = r["rss"][np.searchsorted(sample, g_idx)]
    assert r_best <= r["rss"].min() * (1 + 1e-5)


@pytest.mark.parametrize("pipelined", [False, True])
def test_host_event_runner_equals_device_scan(ctx, pipelined):
    """The end-to-end path from pinned host buffers (copies in, every partition, the selected seed
    and RSS written by the DCA launch straight into the result arrays, copies out) gives the same
    best seed and RSS per partition and the same final hit mask as the device-resident scan, one
    partition at a time and with the next partition's recording beside the DCA."""
    events = [synth.multi_turn_event(i, counts=(4, 8, 8, 16)) for i in range(3)]
    dtype, stride, lam = torch.float32, 32, 1e-2
    field = B.DeviceField.from_synth(UNIFORM)
    S = max(sp.n_seeds for ev in events for sp in ev.partitions)
    n_rec = max(n // stride + 1 for ev in events for n in ev.n_steps)
    H = max(ev.n_hits for ev in events)
    ws = scan.Workspace(S, n_rec, H, dtype)
    ref = []
    for ev in events:
        dev = scan.DeviceEvent.from_event(ev, dtype)
        parts = scan.scan_event(ctx, field, ev, dev, ws, dtype, stride, lam, collect=True)
        ref.append((parts, dev.mask[: ev.n_hits].cpu().numpy().copy()))
    pipe = scan.PipelinedScanner(ctx, field, S, n_rec, H, dtype) if pipelined else None
    runner = scan.HostEventRunner(ctx, field, ws, max(ev.n_wires for ev in events), H, dtype,
                                  pipeline=pipe)
    try:
        outs = []
        for ev in events:           # enqueued back to back, results read once at the end
            out = runner.result_slots()
            runner.run(ev, runner.pin(ev, dtype), stride, lam, out=out)
            outs.append(out)
        torch.cuda.synchronize()
    finally:
        if pipe is not None:
            pipe.close()
    for ev, (parts, mask), (h_idx, h_rss, h_mask) in zip(events, ref, outs):
        n = len(ev.partitions)
        assert [int(v) for v in h_idx[:n]] == [p["idx"] for p in parts]
        assert [float(v) for v in h_rss[:n]] == [p["rss"] for p in parts]
        assert np.array_equal(h_mask[: ev.n_hits].numpy(), mask)
