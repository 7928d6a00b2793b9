"""Iterative refinement (Sec. 2.1): sparse reference seeds and finer lattices around them.

CPU: the oracle's greedy reference walk against the properties that define it (kept references
pairwise non-overlapping; every skipped candidate overlaps a kept one earlier in the order; at most
K; invalid indices skipped; phi compared modulo 2 pi) and the refined lattices against independent
meshgrid constructions.  GPU: the library's references and refined lattices against the oracle's,
and a two-level refinement that ends at a seed at least as good as the coarse scan's best.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1911_09340_gb300 import synth


def _overlap(a, b, hw):
    d = np.array(a, float) - np.array(b, float)
    d[1] = math.remainder(d[1], 2 * math.pi)
    return bool(np.all(np.abs(d) < 2 * np.asarray(hw)))


def _coords(seed):
    return np.array([seed[2], math.atan2(seed[4], seed[3]), seed[5], math.hypot(seed[3], seed[4])])


def _random_seeds(rng, n):
    z = rng.uniform(-0.1, 0.1, n)
    ph = rng.uniform(-math.pi, math.pi, n)
    pz = rng.uniform(10, 20, n)
    pt = rng.uniform(95, 105, n)
    return np.stack([np.zeros(n), np.zeros(n), z, pt * np.cos(ph), pt * np.sin(ph), pz], axis=1)


@pytest.mark.parametrize("K", [1, 3, 8, 32])
def test_reference_walk_properties(K):
    rng = np.random.default_rng(K)
    seeds = _random_seeds(rng, 400)
    idx = rng.permutation(400)[:150]
    idx[[5, 17]] = [-1, 400]                 # invalid slots are skipped
    hw = (0.03, 0.5, 2.0, 3.0)
    refs = O.refine_refs(seeds, idx, hw, K)
    assert 1 <= refs.shape[0] <= K
    for i in range(refs.shape[0]):
        for j in range(i):
            assert not _overlap(refs[i], refs[j], hw)
    # replay the order: each valid candidate before the K-th reference is kept or overlaps a kept one
    kept = 0
    for s in idx:
        if kept == refs.shape[0]:
            break
        if s < 0 or s >= 400:
            continue
        c = _coords(seeds[s])
        if kept < refs.shape[0] and np.allclose(c, refs[kept], rtol=0, atol=1e-12):   # libm ulps
            kept += 1
        else:
            assert any(_overlap(c, refs[j], hw) for j in range(kept))
    assert kept == refs.shape[0]


def test_reference_walk_small_cases():
    # four candidates on a line in z: 0, 1, 2, 3 cm with half-width 0.6 cm: 0 and 2 clash with
    # nothing kept before them, 1 and 3 overlap their predecessors
    seeds = np.array([[0, 0, z, 100.0, 0.0, 10.0] for z in (0.0, 0.01, 0.02, 0.03)])
    hw = (0.006, 0.1, 1.0, 1.0)
    refs = O.refine_refs(seeds, [0, 1, 2, 3], hw, 4)
    assert np.allclose(refs[:, 0], [0.0, 0.02])
    assert O.refine_refs(seeds, [3, 2, 1, 0], hw, 4)[:, 0].tolist() == pytest.approx([0.03, 0.01])
    assert O.refine_refs(seeds, [0, 1, 2, 3], hw, 1).shape == (1, 4)
    # phi is compared modulo 2 pi: azimuths just either side of +-pi overlap
    a = [0, 0, 0.0, 100 * math.cos(math.pi - 1e-3), 100 * math.sin(math.pi - 1e-3), 10.0]
    b = [0, 0, 0.0, 100 * math.cos(-math.pi + 1e-3), 100 * math.sin(-math.pi + 1e-3), 10.0]
    assert O.refine_refs(np.array([a, b]), [0, 1], (0.01, 0.01, 1.0, 1.0), 2).shape[0] == 1
    assert O.refine_refs(np.array([a]), [-1, 5], (0.01, 0.01, 1.0, 1.0), 2).shape[0] == 0


def test_refined_lattices_are_meshgrids_around_the_references():
    shape = synth.LatticeSpec(vxy=(0.01, -0.02), centre=(0, 0, 0, 0), half_width=(0.004, 0.01, 0.5, 1.0),
                              counts=(2, 4, 4, 2))
    refs = np.array([[-0.3, 0.5, 15.0, 100.0], [-0.25, 0.7, 16.0, 101.0]])
    L = O.lattice_refined(shape, refs, 3)
    S1 = 2 * 4 * 4 * 2
    assert L.shape == (3 * S1, 6)
    for k, c in enumerate([refs[0], refs[1], refs[0]]):
        axes = [np.linspace(cc - h, cc + h, n) for cc, h, n in zip(c, shape.half_width, shape.counts)]
        blk = L[k * S1:(k + 1) * S1]
        got = {tuple(np.round(_coords(s), 12)) for s in blk}
        want = {tuple(np.round([z, ph, pz, pt], 12)) for z in axes[0] for ph in axes[1] for pz in axes[2]
                for pt in axes[3]}
        assert got == want
        assert np.allclose(blk[:, 0], 0.01) and np.allclose(blk[:, 1], -0.02)


# ------------------------------------------------------------------------------------------------
# GPU
# ------------------------------------------------------------------------------------------------

@pytest.mark.gpu
@pytest.mark.parametrize("dtype_name", ["float64", "float32"])
def test_gpu_refs_and_refined_lattice_match_oracle(ctx, dtype_name):
    import torch
    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import scan
    dtype = getattr(torch, dtype_name)
    ev = synth.single_event_fp64()
    spec = ev.partitions[0]
    f = B.DeviceField.from_synth(synth.uniform_field(1.0))
    dev = scan.DeviceEvent.from_event(ev, dtype)
    bp = scan.params_for(spec, ev.n_steps[0], dtype, 1)
    ws = scan.Workspace(spec.n_seeds, bp.n_rec, ev.n_hits, dtype, k=64)
    scan.scan_partition(ctx, f, bp, spec, dev, ws, k=64, update_mask=False)
    spacing = [2 * h / (n - 1) for h, n in zip(spec.half_width, spec.counts)]
    hw = [0.75 * s for s in spacing]
    K = 8
    refs = torch.zeros((K, 4), dtype=torch.float64, device="cuda")
    nref = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.comet_scan_refine_refs(ctx, ws.seeds[:, :spec.n_seeds].contiguous(), ws.idx, hw, K, refs, nref)
    seeds_h = ws.seeds[:, :spec.n_seeds].double().cpu().numpy().T
    o_refs = O.refine_refs(seeds_h, ws.idx.cpu().numpy(), hw, K)
    n = int(nref.item())
    assert n == o_refs.shape[0] and n >= 2
    assert np.allclose(refs[:n].cpu().numpy(), o_refs, rtol=1e-14, atol=1e-14)
    fine = synth.LatticeSpec(vxy=spec.vxy, centre=spec.centre, half_width=tuple(hw), counts=(2, 4, 4, 2))
    S2 = K * 64
    seeds2 = torch.empty((6, S2), dtype=dtype, device="cuda")
    charge2 = torch.empty(S2, dtype=torch.int8, device="cuda")
    B.comet_scan_lattice_refined(ctx, fine, refs, nref, K, seeds2, charge2)
    want = O.lattice_refined(fine, o_refs, K)
    got = seeds2.double().cpu().numpy().T
    tol = 1e-12 if dtype == torch.float64 else 2e-7
    assert np.allclose(got, want.astype(np.float32).astype(np.float64) if dtype == torch.float32 else want,
                       rtol=tol, atol=tol)
    assert (charge2.cpu().numpy() == spec.charge).all()


@pytest.mark.gpu
def test_gpu_two_level_refinement_improves_on_the_coarse_best(ctx):
    import torch
    from paper_1911_09340_gb300 import experiments as X
    ev = synth.single_event_fp64()
    r = X.refine_partition(ctx, ev, 0, torch.float64, stride=1, coarse=(4, 4, 8, 8),
                           fine=(3, 3, 3, 3), levels=2, M=64, K=8)
    # odd counts put each reference itself on its finer lattice (recomputed from its coordinates,
    # hence the rounding allowance), so the best RSS cannot grow from level to level
    for a, b in zip(r["levels"][:-1], r["levels"][1:]):
        assert b["best_rss"] <= a["best_rss"] * (1 + 1e-9)
    assert r["levels"][-1]["seeds"] == 8 * 81
    # every level's selected seed is a scanned seed whose RSS the oracle reproduces
    for lv in r["levels"]:
        op = O.Params(n_steps=ev.n_steps[0], stride=1, lam=1e-2, tol=1e-12)
        o = O.scan(synth.uniform_field(1.0), op, lv["best_seed"][None], ev.partitions[0].charge,
                   O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, np.zeros(ev.n_hits, np.uint8))
        assert o["rss"][0] == pytest.approx(lv["best_rss"], rel=1e-10, abs=1e-14)
