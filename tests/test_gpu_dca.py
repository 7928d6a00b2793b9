"""Parity of DCA finding and the RSS (Algorithm 2, Eq. 1) with the FP64 oracle.

Bars: FP64 DCAs within 1e-9 m and RSS within 1e-10 relative (the paper's own CPU/GPU validation
found < O(1e-12), Sec. 4.1); FP32 DCAs within 2 um (track points within 1 um over one turn plus the
FP32 distance arithmetic) and every RSS within the bound those DCAs imply; n_in identical where no
residual sits within the DCA tolerance of the cutoff.  The oracle takes the inputs the device path
receives (FP32: seeds, wires and drifts rounded to float32).  No statistical allowance: every
compared value must meet its bar.  Covered: both dtypes, small and large seed
counts, ragged seed counts, several wire tiles, hits beyond the shared-memory capacity, misaligned
wire rows, W = 0, all hits masked, the pruned and exact paths.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1911_09340_gb300 import binding as B
from paper_1911_09340_gb300 import synth

from gpu_util import FP32_DCA_TOL, both_params, gpu_dca, per_wire_residual, rss_bound, seen

pytestmark = pytest.mark.gpu

UNIFORM = synth.uniform_field(1.0)


def _event_inputs(ev, stride=1, lam=0.01, tol64=True):
    op, bp = both_params(n_steps=ev.n_steps[0], stride=stride, lam=lam,
                         tol=1e-12 if tol64 else 1e-6)
    return op, bp


def test_fp64_exact_path_matches_oracle(ctx):
    ev = synth.single_event_fp64()
    seeds = O.lattice(ev.partitions[0])[::8]
    op, bp = _event_inputs(ev)
    mask = np.zeros(ev.n_hits, np.uint8)
    g = gpu_dca(ctx, B.DeviceField.from_synth(UNIFORM), bp, seeds, -1, ev.wires, ev.hit_offsets,
                ev.drift, mask, torch.float64, want_dca=True)
    r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, mask,
               want_dca=True)
    assert np.abs(g["dca"] - r["dca"]).max() <= 1e-9
    assert np.allclose(g["rss"], r["rss"], rtol=1e-10, atol=0)
    assert np.array_equal(g["n_in"], r["n_in"])
    assert g["n_unconv"] == int(r["n_unconv"].sum())


def test_fp64_pruned_path_equals_exact_path(ctx):
    ev = synth.single_event_fp64()
    seeds = O.lattice(ev.partitions[1])[::8]
    op, bp = _event_inputs(ev)
    mask = np.zeros(ev.n_hits, np.uint8)
    mask[::5] = 1
    f = B.DeviceField.from_synth(UNIFORM)
    a = gpu_dca(ctx, f, bp, seeds, -1, ev.wires, ev.hit_offsets, ev.drift, mask, torch.float64, True)
    b = gpu_dca(ctx, f, bp, seeds, -1, ev.wires, ev.hit_offsets, ev.drift, mask, torch.float64, False)
    assert np.array_equal(a["rss"], b["rss"])
    assert np.array_equal(a["n_in"], b["n_in"])
    r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, mask)
    assert np.allclose(b["rss"], r["rss"], rtol=1e-10, atol=0)


def _fp32_check(g, r, ev_offs, drift, mask, lam, delta=FP32_DCA_TOL):
    """Every DCA of a wire within 3 cm within delta of the oracle's, every RSS within the bound
    those DCAs imply, n_in identical for seeds with no residual within delta of the cutoff."""
    near = r["dca"] < 0.03
    dd = np.abs(g["dca"] - r["dca"])[near]
    assert dd.max() <= delta, (int((dd > delta).sum()), dd.max())
    e = per_wire_residual(r["dca"], ev_offs, drift, mask)
    bound = rss_bound(e, lam, delta)
    excess = np.abs(g["rss"] - r["rss"]) - bound
    assert excess.max() <= 1e-12, (int((excess > 1e-12).sum()), int(np.argmax(excess)))
    edge = (np.abs(e - lam) < delta).any(1)
    assert np.array_equal(g["n_in"][~edge], r["n_in"][~edge])


@pytest.mark.parametrize("stride", [1, 4, 16, 24, 32])
def test_fp32_matches_oracle_multi_turn_event(ctx, stride):
    ev = synth.multi_turn_event(0)
    seeds = O.lattice(ev.partitions[0])[::64].astype(np.float32).astype(np.float64)  # 4096 seeds
    op, bp = both_params(n_steps=ev.n_steps[0], stride=stride, lam=0.01, tol=1e-6)
    op.tol = 1e-12
    mask = np.zeros(ev.n_hits, np.uint8)
    w32, d32 = seen(ev.wires, torch.float32), seen(ev.drift, torch.float32)
    g = gpu_dca(ctx, B.DeviceField.from_synth(UNIFORM), bp, seeds, -1, ev.wires, ev.hit_offsets,
                ev.drift, mask, torch.float32, want_dca=True)
    r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(w32), ev.hit_offsets, d32, mask, want_dca=True)
    _fp32_check(g, r, ev.hit_offsets, d32, mask, 0.01)
    # the pruned path gives the same RSS as the exact path up to FP32 summation of equal terms
    p = gpu_dca(ctx, B.DeviceField.from_synth(UNIFORM), bp, seeds, -1, ev.wires, ev.hit_offsets,
                ev.drift, mask, torch.float32, want_dca=False)
    assert np.allclose(p["rss"], g["rss"], rtol=1e-6, atol=0)
    assert np.array_equal(p["n_in"], g["n_in"])
    # search bounds written by propagate or built by dca itself: the same results
    q = gpu_dca(ctx, B.DeviceField.from_synth(UNIFORM), bp, seeds, -1, ev.wires, ev.hit_offsets,
                ev.drift, mask, torch.float32, want_dca=False, use_bounds=False)
    assert np.array_equal(q["rss"], p["rss"]) and np.array_equal(q["n_in"], p["n_in"])


def test_fp32_large_seed_count_sampled(ctx):
    """65,573 seeds (ragged tail); the oracle checks a sample of them."""
    ev = synth.multi_turn_event(1)
    all_seeds = O.lattice(ev.partitions[0]).astype(np.float32).astype(np.float64)
    seeds = all_seeds[:65573]
    op, bp = both_params(n_steps=ev.n_steps[0], stride=2, lam=0.01, tol=1e-6)
    op.tol = 1e-12
    mask = np.zeros(ev.n_hits, np.uint8)
    g = gpu_dca(ctx, B.DeviceField.from_synth(UNIFORM), bp, seeds, -1, ev.wires, ev.hit_offsets,
                ev.drift, mask, torch.float32, want_dca=False)
    sample = np.unique(np.concatenate([np.arange(0, 65573, 61), [65572, int(np.argmin(g["rss"]))]]))
    w32, d32 = seen(ev.wires, torch.float32), seen(ev.drift, torch.float32)
    r = O.scan(UNIFORM, op, seeds[sample], -1, O.wires_aos(w32), ev.hit_offsets, d32, mask,
               want_dca=True)
    e = per_wire_residual(r["dca"], ev.hit_offsets, d32, mask)
    bound = rss_bound(e, 0.01, FP32_DCA_TOL)
    excess = np.abs(g["rss"][sample] - r["rss"]) - bound
    assert excess.max() <= 1e-12, (int((excess > 1e-12).sum()), sample[int(np.argmax(excess))])


def _many_wires_case(n_wires=600, hits_per_wire=3, seed=5):
    ch = synth.make_chamber()
    ev = synth.single_event_fp64(ch)
    rng = np.random.default_rng(seed)
    extra = rng.choice(ch.n_wires, size=n_wires - ev.n_wires, replace=False)
    ids = np.unique(np.concatenate([ev.wire_ids, extra]))[:n_wires]
    wires = np.concatenate([ch.a[:, ids], ch.u[:, ids]], axis=0)
    offs = np.arange(len(ids) + 1, dtype=np.int32) * hits_per_wire
    drift = rng.uniform(0, 8e-3, size=offs[-1])
    mask = (rng.uniform(size=offs[-1]) < 0.2).astype(np.uint8)
    return ev, wires, offs, drift, mask


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("misalign", [0, 1, 3])
def test_many_wires_many_hits_misaligned(ctx, dtype, misalign):
    ev, wires, offs, drift, mask = _many_wires_case()
    assert wires.shape[1] > 2 * 256 and offs[-1] > 1024     # several tiles, hits read from global
    seeds = O.lattice(ev.partitions[0])[::97].astype(np.float32).astype(np.float64)
    op, bp = both_params(n_steps=ev.n_steps[0], lam=0.01,
                         tol=1e-12 if dtype == torch.float64 else 1e-6)
    op.tol = 1e-12
    for want in (True, False):
        g = gpu_dca(ctx, B.DeviceField.from_synth(UNIFORM), bp, seeds, -1, wires, offs, drift, mask,
                    dtype, want_dca=want, misalign=misalign)
        r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(seen(wires, dtype)), offs, seen(drift, dtype),
                   mask, want_dca=True)
        if dtype == torch.float64:
            if want:
                # wires metres away whose closest recorded state is a track end: the refinement
                # extrapolates with metre-long RK4 steps, where rounding order decides the result
                # (they are capped at lambda either way); near wires must agree to 1e-9 m
                near = r["dca"] < 0.05
                assert np.abs(g["dca"] - r["dca"])[near].max() <= 1e-9
            assert np.allclose(g["rss"], r["rss"], rtol=1e-10, atol=0)
            assert np.array_equal(g["n_in"], r["n_in"])
        else:
            if want:
                near = r["dca"] < 0.05
                assert np.abs(g["dca"] - r["dca"])[near].max() <= FP32_DCA_TOL
            e = per_wire_residual(r["dca"], offs, seen(drift, dtype), mask)
            bound = rss_bound(e, 0.01, FP32_DCA_TOL)
            excess = np.abs(g["rss"] - r["rss"]) - bound
            assert excess.max() <= 1e-12, (int((excess > 1e-12).sum()), int(np.argmax(excess)))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_degenerate_inputs(ctx, dtype):
    ev = synth.single_event_fp64()
    seeds = O.lattice(ev.partitions[0])[:5]
    op, bp = both_params(n_steps=ev.n_steps[0], tol=1e-12 if dtype == torch.float64 else 1e-6)
    f = B.DeviceField.from_synth(UNIFORM)
    # no wires at all
    g = gpu_dca(ctx, f, bp, seeds, -1, np.zeros((6, 0)), np.zeros(1, np.int32), np.zeros(0),
                np.zeros(0, np.uint8), dtype, want_dca=False)
    assert np.all(g["rss"] == 0) and np.all(g["n_in"] == 0)
    # every hit masked: no wire is in the sum
    mask = np.ones(ev.n_hits, np.uint8)
    g = gpu_dca(ctx, f, bp, seeds, -1, ev.wires, ev.hit_offsets, ev.drift, mask, dtype, want_dca=True)
    assert np.all(g["rss"] == 0) and np.all(g["n_in"] == 0)
    r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(seen(ev.wires, dtype)), ev.hit_offsets,
               seen(ev.drift, dtype), mask, want_dca=True)
    tol = 1e-9 if dtype == torch.float64 else FP32_DCA_TOL
    assert np.abs(g["dca"] - r["dca"])[r["dca"] < 0.03].max() <= tol
    # a single seed
    g = gpu_dca(ctx, f, bp, seeds[:1], -1, ev.wires, ev.hit_offsets, ev.drift,
                np.zeros(ev.n_hits, np.uint8), dtype, want_dca=False)
    z = np.zeros(ev.n_hits, np.uint8)
    r = O.scan(UNIFORM, op, seeds[:1], -1, O.wires_aos(seen(ev.wires, dtype)), ev.hit_offsets,
               seen(ev.drift, dtype), z, want_dca=True)
    if dtype == torch.float64:
        assert np.allclose(g["rss"], r["rss"], rtol=1e-10, atol=0)
    else:
        e = per_wire_residual(r["dca"], ev.hit_offsets, seen(ev.drift, dtype), z)
        assert np.abs(g["rss"] - r["rss"]).max() <= rss_bound(e, op.lam, FP32_DCA_TOL).max() + 1e-12


def test_unconverged_count_matches_oracle(ctx):
    ev = synth.single_event_fp64()
    seeds = O.lattice(ev.partitions[0])[::64]
    op, bp = both_params(n_steps=ev.n_steps[0], stride=5, max_iter=1)
    mask = np.zeros(ev.n_hits, np.uint8)
    g = gpu_dca(ctx, B.DeviceField.from_synth(UNIFORM), bp, seeds, -1, ev.wires, ev.hit_offsets,
                ev.drift, mask, torch.float64, want_dca=True)
    r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, mask,
               want_dca=True)
    assert int(r["n_unconv"].sum()) > 0
    assert g["n_unconv"] == int(r["n_unconv"].sum())
    assert np.abs(g["dca"] - r["dca"]).max() <= 1e-9


@pytest.mark.parametrize("interleaved", [False, True])
def test_table_field_dca(ctx, interleaved):
    field = synth.table_field(spacing=0.02)
    ev = synth.single_event_fp64()
    seeds = O.lattice(ev.partitions[0])[::33]
    op, bp = both_params(n_steps=ev.n_steps[0])
    mask = np.zeros(ev.n_hits, np.uint8)
    g = gpu_dca(ctx, B.DeviceField.from_synth(field, interleaved=interleaved), bp, seeds, -1, ev.wires,
                ev.hit_offsets, ev.drift, mask, torch.float64, want_dca=True)
    r = O.scan(field, op, seeds, -1, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, mask,
               want_dca=True)
    assert np.abs(g["dca"] - r["dca"]).max() <= 1e-9
    assert np.allclose(g["rss"], r["rss"], rtol=1e-10, atol=0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_interleaved_table_is_bit_identical(ctx, dtype):
    """Field kind 2 ([nz][ny][nx][4]) interpolates the same values in the same order as kind 1."""
    field = synth.table_field(spacing=0.02)
    ev = synth.single_event_fp64()
    seeds = O.lattice(ev.partitions[0])[::17]
    _, bp = both_params(n_steps=ev.n_steps[0], stride=4)
    mask = np.zeros(ev.n_hits, np.uint8)
    outs = [gpu_dca(ctx, B.DeviceField.from_synth(field, interleaved=il), bp, seeds, -1, ev.wires,
                    ev.hit_offsets, ev.drift, mask, dtype, want_dca=True) for il in (False, True)]
    for k in ("rss", "dca", "n_in"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("use_bounds", [True, False])
def test_pruned_search_keeps_wires_beyond_the_track_ends(ctx, dtype, use_bounds):
    """Wires crossing the track's extension 0.875 of an interval past its last recorded state and
    before its first: the refinement from the end state reaches them (DCA ~0.4-1 mm), although the
    closest recorded state is ~14 mm away, beyond cap + h_rec/2.  The pruned path (segment spheres
    from propagate or built by the DCA kernel) must still refine those pairs."""
    from gpu_util import per_wire_residual, rss_bound
    from track_ends import end_case
    seeds, wires, offs, drift, n = end_case(UNIFORM)
    lam = 2e-3
    f64 = dtype == torch.float64
    op, bp = both_params(n_steps=n, stride=16, lam=lam, tol=1e-12 if f64 else 1e-6)
    mask = np.zeros(3, np.uint8)
    g = gpu_dca(ctx, B.DeviceField.from_synth(UNIFORM), bp, seeds, -1, wires, offs, drift, mask, dtype,
                want_dca=False, use_bounds=use_bounds)
    r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(seen(wires, dtype)), offs, seen(drift, dtype),
               mask, want_dca=True)
    assert (np.abs(r["dca"][:, :2] - drift[:2]) < lam).all()   # the end wires are inliers in the oracle
    if f64:
        assert np.allclose(g["rss"], r["rss"], rtol=1e-10, atol=0)
    else:
        e = per_wire_residual(r["dca"], offs, seen(drift, dtype), mask)
        assert (np.abs(g["rss"] - r["rss"]) <= rss_bound(e, lam, FP32_DCA_TOL) + 1e-12).all()
    assert np.array_equal(g["n_in"], r["n_in"])


def _wires_case(n_wires, hits_per_wire=3, seed=7):
    """The event's own wires first, then random chamber wires, n_wires in all; random drifts."""
    ch = synth.make_chamber()
    ev = synth.single_event_fp64(ch)
    rng = np.random.default_rng(seed)
    own = np.sort(np.asarray(ev.wire_ids))
    if n_wires <= own.size:
        ids = own[:n_wires]
    else:
        rest = np.setdiff1d(np.arange(ch.n_wires), own)
        ids = np.concatenate([own, rng.choice(rest, size=n_wires - own.size, replace=False)])
    wires = np.concatenate([ch.a[:, ids], ch.u[:, ids]], axis=0)
    offs = np.arange(ids.size + 1, dtype=np.int32) * hits_per_wire
    drift = rng.uniform(0, 8e-3, size=offs[-1])
    mask = (rng.uniform(size=offs[-1]) < 0.2).astype(np.uint8)
    return ev, wires, offs, drift, mask


@pytest.mark.parametrize("n_wires", [1, 32, 33, 64, 65, 1024, 1025])
def test_wire_chunk_boundaries(ctx, n_wires):
    """Each seed's sum is cut into chunks of at most 32 wires, one work item per (32-seed group,
    chunk), the chunk sums added in chunk order; W = 1025 takes the tiled kernel instead.  At the
    chunk boundaries: FP64 RSS within the bound that the 1e-9 m DCA bar implies term by term (a
    single small residual makes any relative bar meaningless) plus the summation order, n_in equal
    away from the cutoff, pruned and exact paths; and FP32 sums bit-identical from run to run (no
    dependence on which warp finishes a group last)."""
    ev, wires, offs, drift, mask = _wires_case(n_wires)
    assert wires.shape[1] == n_wires
    seeds = O.lattice(ev.partitions[0])[::7].astype(np.float32).astype(np.float64)   # 586 seeds
    f = B.DeviceField.from_synth(UNIFORM)
    lam = 0.01
    op, bp = both_params(n_steps=ev.n_steps[0], stride=16, lam=lam, tol=1e-12)
    r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(wires), offs, drift, mask, want_dca=True)
    e = per_wire_residual(r["dca"], offs, drift, mask)
    bound = rss_bound(e, lam, 1e-9, fp32=False) + 1e-14 * r["rss"]
    edge = (np.abs(e - lam) < 1e-9).any(1)
    for want in (True, False):
        g = gpu_dca(ctx, f, bp, seeds, -1, wires, offs, drift, mask, torch.float64, want_dca=want)
        assert (np.abs(g["rss"] - r["rss"]) <= bound).all()
        assert np.array_equal(g["n_in"][~edge], r["n_in"][~edge])
    _, bp32 = both_params(n_steps=ev.n_steps[0], stride=16, lam=0.01, tol=1e-6)
    a = gpu_dca(ctx, f, bp32, seeds, -1, wires, offs, drift, mask, torch.float32, want_dca=False)
    b = gpu_dca(ctx, f, bp32, seeds, -1, wires, offs, drift, mask, torch.float32, want_dca=False)
    assert np.array_equal(a["rss"], b["rss"]) and np.array_equal(a["n_in"], b["n_in"])


@pytest.mark.parametrize("chunk_wires", [4, 16, 100])
def test_chunk_width_setting_keeps_the_oracle_sums(ctx, chunk_wires):
    """The context's wires per chunk (4, 16 and 100; 200 wires, 586 seeds): FP64 RSS within the
    bound of the 1e-9 m DCA bar and n_in identical away from the cutoff; FP32 RSS within the bound
    of the 2 um bar."""
    ev, wires, offs, drift, mask = _wires_case(200)
    seeds = O.lattice(ev.partitions[0])[::7].astype(np.float32).astype(np.float64)
    f = B.DeviceField.from_synth(UNIFORM)
    lam = 0.01
    c = B.Context(0)
    try:
        c.set_dca_chunk_wires(chunk_wires)
        for dtype, delta in ((torch.float64, 1e-9), (torch.float32, FP32_DCA_TOL)):
            op, bp = both_params(n_steps=ev.n_steps[0], stride=16, lam=lam,
                                 tol=1e-12 if dtype == torch.float64 else 1e-6)
            op.tol = 1e-12
            r = O.scan(UNIFORM, op, seeds, -1, O.wires_aos(seen(wires, dtype)), offs,
                       seen(drift, dtype), mask, want_dca=True)
            e = per_wire_residual(r["dca"], offs, seen(drift, dtype), mask)
            bound = rss_bound(e, lam, delta, fp32=dtype == torch.float32) + 1e-14 * r["rss"]
            g = gpu_dca(c, f, bp, seeds, -1, wires, offs, drift, mask, dtype, want_dca=False)
            assert (np.abs(g["rss"] - r["rss"]) <= bound + 1e-12).all()
            edge = (np.abs(e - lam) < delta).any(1)
            assert np.array_equal(g["n_in"][~edge], r["n_in"][~edge])
    finally:
        c.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n_wires", [200, 1025])
def test_copy_wait_give_up_falls_back_to_plain_loads(ctx, dtype, n_wires):
    """With the context's copy wait set to 0, every bulk-copy wait of the DCA kernels gives up at
    once: the kernel re-reads the staged arrays with plain loads, sets status bit 0, and waits
    (bounded) for the abandoned copy before its shared memory is reused.  Results are bit-identical
    to a normal run: 200 wires with 600 hits (persistent kernel, hits staged) and 1025 wires (tiled
    kernel, staged tile by tile)."""
    ev, wires, offs, drift, mask = _wires_case(n_wires)
    seeds = O.lattice(ev.partitions[0])[::13].astype(np.float32).astype(np.float64)
    f = B.DeviceField.from_synth(UNIFORM)
    _, bp = both_params(n_steps=ev.n_steps[0], stride=16, lam=0.01,
                        tol=1e-12 if dtype == torch.float64 else 1e-6)
    ref = gpu_dca(ctx, f, bp, seeds, -1, wires, offs, drift, mask, dtype, want_dca=False)
    c0 = B.Context(0)
    try:
        assert c0.status() == 0
        c0.set_copy_wait(0)
        got = gpu_dca(c0, f, bp, seeds, -1, wires, offs, drift, mask, dtype, want_dca=False)
        assert c0.status() & 1
        for k in ("rss", "n_in"):
            assert np.array_equal(got[k], ref[k]), k
        c0.set_copy_wait(2_000_000_000)
    finally:
        c0.close()
