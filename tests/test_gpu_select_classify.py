"""Parity of selection (Sec. 2.1, top-k) and classification (Sec. 2.1, 3.1) with the oracle.

Selection is index work: bit-exact.  Classification is bit-identical except for hits whose residual
|D - r| lies within 1 um (FP32; 1e-9 m FP64) of lambda.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1911_09340_gb300 import binding as B
from paper_1911_09340_gb300 import synth

from gpu_util import CLASS_EDGE, FP32_DCA_TOL, both_params, dev_wires, gpu_propagate, seen

pytestmark = pytest.mark.gpu
UNIFORM = synth.uniform_field(1.0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("S", [1, 2, 2047, 2049, 70001, 1 << 18])
def test_select_matches_oracle(ctx, dtype, S):
    rng = np.random.default_rng(S)
    v = rng.integers(0, 50, size=S).astype(np.float64) * 0.125      # many exact ties
    if S > 10:
        v[rng.integers(0, S, size=5)] = np.nan
    v = v.astype(np.float32 if dtype == torch.float32 else np.float64).astype(np.float64)
    rss = torch.as_tensor(v, dtype=dtype, device="cuda")
    for k in sorted({1, min(10, S), min(64, S)}):
        idx = torch.full((k,), -7, dtype=torch.int64, device="cuda")
        val = torch.zeros(k, dtype=dtype, device="cuda")
        B.comet_scan_select(ctx, rss, k, idx, val)
        ri, rv = O.select(v, k)
        assert np.array_equal(idx.cpu().numpy(), ri)
        assert np.array_equal(val.double().cpu().numpy(), rv, equal_nan=True)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("case", ["event", "ties", "ragged", "single", "no_wires", "tiled", "exact"])
def test_selection_inside_the_dca_launch_equals_select(ctx, dtype, case):
    """comet_scan_dca's optional best_idx / best_rss (the k = 1 selection folded into the DCA
    launch: per warp, per CTA, then the last CTA) equal comet_scan_select(k = 1) on the RSS the same
    launch wrote, bit for bit: an event's partition (persistent kernel), seeds duplicated so that
    equal RSS values tie (lowest index wins), a ragged seed count, one seed, no wires (every RSS 0:
    seed 0),
    and more than 1024 wires (tiled kernel, one CTA per 128 seeds), and the exhaustive path that a
    requested dca_out takes (every wire refined from the closest of all states)."""
    from gpu_util import gpu_propagate
    ev = synth.multi_turn_event(1, counts=(4, 8, 8, 16))
    seeds = O.lattice(ev.partitions[0])
    wires, offs, drift = ev.wires, ev.hit_offsets, ev.drift
    if case == "ties":
        seeds = np.concatenate([seeds[::2], seeds[::2], seeds[4:5]])   # every seed twice, in order
    elif case == "ragged":
        seeds = seeds[:3001]
    elif case == "single":
        seeds = seeds[1000:1001]
    elif case == "no_wires":
        wires, offs, drift = np.zeros((6, 0)), np.zeros(1, np.int32), np.zeros(0)
    elif case == "tiled":
        ch = synth.make_chamber()
        ids = np.arange(1100) * 3
        wires = np.concatenate([ch.a[:, ids], ch.u[:, ids]], axis=0)
        offs = np.arange(1101, dtype=np.int32)
        drift = np.random.default_rng(2).uniform(0, 8e-3, size=1100)
    _, bp = both_params(n_steps=ev.n_steps[0], stride=32, lam=0.01,
                        tol=1e-12 if dtype == torch.float64 else 1e-6)
    f = B.DeviceField.from_synth(UNIFORM)
    _, charge, pts, nv = gpu_propagate(ctx, f, bp, seeds, -1, dtype)
    S, W = seeds.shape[0], wires.shape[1]
    w = dev_wires(wires, dtype)
    o = torch.as_tensor(np.asarray(offs, np.int32), device="cuda")
    d = torch.as_tensor(np.asarray(drift), dtype=dtype, device="cuda")
    m = torch.zeros(max(int(offs[-1]), 1), dtype=torch.uint8, device="cuda")
    rss = torch.empty(S, dtype=dtype, device="cuda")
    n_in = torch.empty(S, dtype=torch.int32, device="cuda")
    for rep in range(2):                  # twice: the arrival counter is left at zero
        bi = torch.full((1,), -5, dtype=torch.int64, device="cuda")
        bv = torch.full((1,), -5.0, dtype=dtype, device="cuda")
        dca = torch.empty((max(W, 1), S), dtype=dtype, device="cuda") if case == "exact" else None
        B.comet_scan_dca(ctx, f, bp, pts, nv, charge, w, o, d, m, rss, n_in, n_wires=W, dca_out=dca,
                         best_idx=bi, best_rss=bv)
        ri = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        rv = torch.zeros(1, dtype=dtype, device="cuda")
        B.comet_scan_select(ctx, rss, 1, ri, rv)
        torch.cuda.synchronize()
        assert int(bi[0]) == int(ri[0]) and bv.cpu().numpy()[0] == rv.cpu().numpy()[0]
        r = rss.double().cpu().numpy()
        assert int(bi[0]) == int(np.flatnonzero(r == r.min())[0])
    if case == "ties":
        assert int(bi[0]) < S // 2 + 1 and r[int(bi[0])] == r[int(bi[0]) + (S - 1) // 2]
    if case == "no_wires":
        assert int(bi[0]) == 0 and float(bv[0]) == 0.0


def test_select_rejects_bad_k(ctx):
    rss = torch.zeros(10, dtype=torch.float32, device="cuda")
    idx = torch.zeros(65, dtype=torch.int64, device="cuda")
    for k in (0, 11, 65):
        with pytest.raises(B.CometError):
            B.comet_scan_select(ctx, rss, k, idx)


def _classify_case(ctx, dtype, ev, part, seed_idx, mask):
    spec = ev.partitions[part]
    seeds = O.lattice(spec)
    if dtype == torch.float32:
        seeds = seeds.astype(np.float32).astype(np.float64)
    op, bp = both_params(n_steps=ev.n_steps[part], tol=1e-12 if dtype == torch.float64 else 1e-6)
    op.tol = 1e-12
    sub = seeds[max(0, seed_idx - 40): seed_idx + 41]
    local = seed_idx - max(0, seed_idx - 40)
    f = B.DeviceField.from_synth(UNIFORM)
    _, charge, pts, nv = gpu_propagate(ctx, f, bp, sub, -1, dtype)
    W, H = ev.n_wires, ev.n_hits
    w = dev_wires(ev.wires, dtype)
    o = torch.as_tensor(ev.hit_offsets, device="cuda")
    d = torch.as_tensor(ev.drift, dtype=dtype, device="cuda")
    m = torch.as_tensor(mask, device="cuda")
    si = torch.tensor([local], dtype=torch.int64, device="cuda")
    hc = torch.full((H,), 7, dtype=torch.uint8, device="cuda")
    dw = torch.full((W,), float("nan"), dtype=dtype, device="cuda")
    B.comet_scan_classify(ctx, f, bp, pts, nv, charge, si, w, o, d, m, hc, dca_wire=dw,
                          update_mask=True, n_wires=W)
    cls, dwr, m2 = O.classify(UNIFORM, op, sub[local], -1, O.wires_aos(seen(ev.wires, dtype)),
                              ev.hit_offsets, seen(ev.drift, dtype), mask, update_mask=True)
    return hc.cpu().numpy(), dw.double().cpu().numpy(), m.cpu().numpy(), cls, dwr, m2, op.lam


@pytest.mark.parametrize("dtype,delta", [(torch.float64, 1e-9), (torch.float32, FP32_DCA_TOL)])
def test_classify_matches_oracle(ctx, dtype, delta):
    """Hit classes of three seeds with every 7th hit masked: bit-identical to the oracle's except
    hits whose residual lies within the classification band (1 um FP32, 1e-9 m FP64) of lambda;
    the seed's DCA to every wire within the DCA bar; the mask update is the OR of the classes."""
    ev = synth.multi_turn_event(2)
    mask = np.zeros(ev.n_hits, np.uint8)
    mask[::7] = 1
    wid = np.repeat(np.arange(ev.n_wires), np.diff(ev.hit_offsets))
    d = seen(ev.drift, dtype)
    for seed_idx in (0, 12345, (1 << 18) - 1):
        hc, dw, m, cls, dwr, m2, lam = _classify_case(ctx, dtype, ev, 0, seed_idx, mask)
        near = dwr < 0.03
        assert np.abs(dw - dwr)[near].max() <= delta
        e = np.abs(dwr[wid] - d)
        edge = np.abs(e - lam) < CLASS_EDGE[dtype]
        diff = np.flatnonzero(hc != cls)
        assert np.all(edge[diff]), (seed_idx, diff[~edge[diff]])
        assert np.array_equal(m, np.maximum(mask, hc))
        assert set(np.unique(hc)) <= {0, 1}


def test_classify_out_of_range_index_sets_status():
    ctx = B.Context(0)     # a fresh context: this test sets a status bit on purpose
    ev = synth.single_event_fp64()
    seeds = O.lattice(ev.partitions[0])[:4]
    op, bp = both_params(n_steps=ev.n_steps[0])
    f = B.DeviceField.from_synth(UNIFORM)
    _, charge, pts, nv = gpu_propagate(ctx, f, bp, seeds, -1, torch.float64)
    w = dev_wires(ev.wires, torch.float64)
    o = torch.as_tensor(ev.hit_offsets, device="cuda")
    d = torch.as_tensor(ev.drift, dtype=torch.float64, device="cuda")
    m = torch.zeros(ev.n_hits, dtype=torch.uint8, device="cuda")
    hc = torch.full((ev.n_hits,), 9, dtype=torch.uint8, device="cuda")
    si = torch.tensor([4], dtype=torch.int64, device="cuda")
    B.comet_scan_classify(ctx, f, bp, pts, nv, charge, si, w, o, d, m, hc, n_wires=ev.n_wires)
    assert ctx.status() & 2
    assert int(hc.sum()) == 0 and int(m.sum()) == 0
    ctx.close()
