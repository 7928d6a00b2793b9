"""Studies built on the scan (the evaluation side of the paper's Sec. 3, on synthetic events).

    python -m paper_1911_09340_gb300.experiments lambda-sweep [--events N] [--stride s]
    python -m paper_1911_09340_gb300.experiments backward [--events N] [--stride s]
    python -m paper_1911_09340_gb300.experiments iterative [--events N] [--stride s]
    python -m paper_1911_09340_gb300.experiments gauss-newton [--events N] [--lambda-mm 0.8]
    python -m paper_1911_09340_gb300.experiments batch [--events N]
    python -m paper_1911_09340_gb300.experiments table-field [--events N]
    python -m paper_1911_09340_gb300.experiments single-event [--reps N] [--stride s]

* ``lambda-sweep``: hit-classification efficiency and purity (metrics.py) of the first stage and of
  all stages as the cutoff lambda runs over 0.5-1.2 mm in 0.1 mm steps (the range of the paper's
  cutoff optimisation, Sec. 3.2; there the first stage is the last turn, here it is the first turn
  from the vertex, and there is no DAF fit or self-refining after the scan).
* ``backward``: the first stage scanned forwards from the start of the turn and backwards from its
  end with the charge and momentum flipped (the paper's two half tracks, Sec. 3.1), each over the
  whole turn.
* ``iterative``: the dense 2^18-seed grid against an iterative scan (Sec. 2.1: sparse low-RSS
  references, finer lattices around them) of a 2^14 coarse grid refined twice.
* ``gauss-newton``: the dense grid against Gauss-Newton on the smoothed RSS (comet_scan_jacobian,
  comet_scan_gn_step) started from the top 16 seeds of a 2^14 grid.
* ``batch``: events/s and per-event latency of many uneven events, per-event path against
  continuous batching (batch.py) under the autotuned configuration.
* ``table-field``: evaluations/s on the non-uniform (tabulated solenoid) field workload, with the
  uniform-field path on the same events beside it.
* ``single-event``: the small single-event configuration (2 partitions of 8^4 seeds) in FP64 and
  FP32: time per event and the DCA kernel's algorithmic flop rate against the FP64 and FP32 rates.

Every scan runs through the library's kernels (scan.scan_partition); only the metrics are computed
on the host from the copied-back hit classes.  One JSON line per result.
"""
from __future__ import annotations

import argparse
import json
import sys
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B
from . import metrics as M
from . import scan, synth


def scan_stages(ctx, field, ev, dev, ws, specs: Sequence, n_steps: Sequence[int], dtype, stride: int,
                lam: float) -> List[np.ndarray]:
    """Scans the given partitions of one event in order (hits classified at a stage are masked for
    the next); returns each stage's classified-hit flags."""
    dev.mask.zero_()
    out = []
    for spec, n in zip(specs, n_steps):
        bp = scan.params_for(spec, n, dtype, stride, lam)
        scan.scan_partition(ctx, field, bp, spec, dev, ws)
        out.append(ws.hit_class[: max(ev.n_hits, 1)].cpu().numpy()[: ev.n_hits].astype(bool))
    return out


def _setup(events, dtype, stride):
    ctx = B.Context(torch.cuda.current_device())
    field = B.DeviceField.from_synth(synth.uniform_field(1.0))
    S = max(sp.n_seeds for ev in events for sp in ev.partitions)
    n_rec = max(n // stride + 1 for ev in events for n in ev.n_steps)
    H = max(ev.n_hits for ev in events)
    ws = scan.Workspace(S, n_rec, H, dtype)
    return ctx, field, ws


def lambda_sweep(n_events: int = 32, lambdas_mm=(0.5, 0.6, 0.7, 0.8, 0.9, 1.0, 1.1, 1.2),
                 stride: int = 16, dtype=torch.float32, counts=(16, 16, 32, 32)):
    events = [synth.multi_turn_event(i, counts=counts) for i in range(n_events)]
    ctx, field, ws = _setup(events, dtype, stride)
    devs = [scan.DeviceEvent.from_event(ev, dtype) for ev in events]
    rows = []
    for lam_mm in lambdas_mm:
        lam = lam_mm * 1e-3
        first, every = [], []
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for ev, dev in zip(events, devs):
            t0.record()
            cls = scan_stages(ctx, field, ev, dev, ws, ev.partitions, ev.n_steps, dtype, stride, lam)
            t1.record()
            t1.synchronize()
            ms += t0.elapsed_time(t1)
            st = M.event_metrics(cls, ev.hit_turn)
            first.append(st[0])
            every.extend(st)
        rows.append({"study": "lambda-sweep", "lambda_mm": lam_mm, "events": n_events,
                     "first_stage": M.average(first), "all_stages": M.average(every),
                     "first_stage_turn0": float(np.mean([s.turn == 0 for s in first])),
                     "ms_per_event": ms / n_events, "stride": stride, "seeds_per_partition":
                     int(np.prod(counts))})
    ctx.close()
    return rows


def backward_study(n_events: int = 32, stride: int = 16, lam: float = 1e-2, dtype=torch.float32,
                   counts=(16, 16, 32, 32)):
    events = [synth.multi_turn_event(i, counts=counts) for i in range(n_events)]
    ctx, field, ws = _setup(events, dtype, stride)
    fwd, bwd = [], []
    for ev in events:
        dev = scan.DeviceEvent.from_event(ev, dtype)
        n = ev.n_steps[0]
        fwd.append(M.stage_metrics(scan_stages(ctx, field, ev, dev, ws, ev.partitions[:1], [n], dtype,
                                               stride, lam)[0], ev.hit_turn))
        back = synth.backward_partition(ev, 0)
        bwd.append(M.stage_metrics(scan_stages(ctx, field, ev, dev, ws, [back], [n], dtype, stride,
                                               lam)[0], ev.hit_turn))
    ctx.close()
    return [{"study": "backward", "events": n_events, "lambda_mm": lam * 1e3, "stride": stride,
             "forward_first_stage": M.average(fwd), "backward_first_stage": M.average(bwd),
             "same_turn": float(np.mean([a.turn == b.turn for a, b in zip(fwd, bwd)]))}]


def _scan_seeds(ctx, field, bp, dev, ws, S, M):
    """propagate -> dca -> select(top M) on the S seeds already in ws.seeds / ws.charge."""
    seeds, charge, pts, nv, rss, n_in = ws.views(S, bp.n_rec)
    bounds = ws.bounds[: (S + 31) // 32]
    B.comet_scan_propagate(ctx, field, bp, seeds, charge, pts, nv, bounds=bounds)
    B.comet_scan_dca(ctx, field, bp, pts, nv, charge, dev.wires, dev.hit_offsets, dev.drift, dev.mask,
                     rss, n_in, n_unconverged=ws.n_unconv, n_wires=dev.W, bounds=bounds)
    B.comet_scan_select(ctx, rss, M, ws.idx[:M], ws.best[:M])


def refine_partition(ctx, ev, part: int, dtype=torch.float32, stride: int = 16, lam: float = 1e-2,
                     coarse=(8, 8, 16, 16), fine=(5, 5, 5, 5), levels: int = 2, M: int = 64,
                     K: int = 16, shrink: float = 0.75, keep_top: int = 0):
    """Iterative scan of one turn partition (Sec. 2.1): a coarse lattice over the prior ranges, then
    ``levels`` rounds of: the top-M seeds -> up to K sparse references (comet_scan_refine_refs) ->
    K lattices of ``fine`` counts around them with half-widths ``shrink`` x the previous spacing
    (comet_scan_lattice_refined) -> scan.  Odd ``fine`` counts keep each reference on its own finer
    lattice and shrink the spacing by 2 x shrink / (count - 1) per level.  Everything stays on the
    device; the per-level best seed and RSS are copied back at the end.  Returns
    {"levels": [...], "ms": total GPU time}."""
    import dataclasses as dc
    spec0 = ev.partitions[part]
    n = ev.n_steps[part]
    field = B.DeviceField.from_synth(synth.uniform_field(1.0))
    dev = scan.DeviceEvent.from_event(ev, dtype)
    bp = scan.params_for(spec0, n, dtype, stride, lam)
    S0 = int(np.prod(coarse))
    S1 = K * int(np.prod(fine))
    ws = scan.Workspace(max(S0, S1), bp.n_rec, ev.n_hits, dtype, k=M)
    refs = torch.zeros((K, 4), dtype=torch.float64, device="cuda")
    nref = torch.zeros(1, dtype=torch.int32, device="cuda")
    coarse_spec = dc.replace(spec0, counts=tuple(coarse))
    best_idx, best_rss, best_seed, sizes, marks = [], [], [], [], []
    t0 = torch.cuda.Event(enable_timing=True)
    t0.record()
    B.comet_scan_lattice(ctx, coarse_spec, ws.seeds.view(-1)[: 6 * S0].view(6, S0), ws.charge[:S0])
    _scan_seeds(ctx, field, bp, dev, ws, S0, M)
    hw = list(coarse_spec.half_width)
    counts = list(coarse)
    S = S0
    for lv in range(levels + 1):
        seeds = ws.seeds.view(-1)[: 6 * S].view(6, S)
        best_idx.append(ws.idx[:1].clone())
        best_rss.append(ws.best[:1].clone())
        best_seed.append(torch.index_select(seeds, 1, ws.idx[:1]).clone())
        sizes.append(S)
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        marks.append(e)
        if lv == levels:
            break
        hw = [shrink * 2.0 * h / (c - 1) if c > 1 else h for h, c in zip(hw, counts)]
        counts = list(fine)
        B.comet_scan_refine_refs(ctx, seeds, ws.idx[:M], hw, K, refs, nref)
        shape = dc.replace(spec0, half_width=tuple(hw), counts=tuple(fine))
        S = S1
        B.comet_scan_lattice_refined(ctx, shape, refs, nref, K, ws.seeds.view(-1)[: 6 * S].view(6, S),
                                     ws.charge[:S])
        _scan_seeds(ctx, field, bp, dev, ws, S, M)
    if keep_top:
        # hand the last level's seeds and top-M indices to the caller (e.g. Gauss-Newton)
        return {"seeds": ws.seeds.view(-1)[: 6 * S].view(6, S), "idx": ws.idx[:M], "nref": nref,
                "ws": ws}
    torch.cuda.synchronize()
    out = []
    prev = t0
    for lv in range(levels + 1):
        out.append({"level": lv, "seeds": sizes[lv], "best_rss": float(best_rss[lv].item()),
                    "best_seed": best_seed[lv][:, 0].double().cpu().numpy(),
                    "ms": prev.elapsed_time(marks[lv])})
        prev = marks[lv]
    return {"levels": out, "ms": t0.elapsed_time(marks[-1])}


def iterative_study(n_events: int = 16, stride: int = 16, lam: float = 1e-2, dtype=torch.float32):
    """Best RSS, momentum error of the best seed against the truth and GPU time: the dense 2^18 grid
    of the benchmark against a coarse 2^14 grid refined twice (16 references, 5^4 seeds each)."""
    ctx = B.Context(torch.cuda.current_device())
    dense, itr = [], []
    for i in range(n_events):
        ev = synth.multi_turn_event(i)
        p_true = float(np.hypot(ev.pt, ev.pz))
        runs = []
        for kw in (dict(coarse=(16, 16, 32, 32), levels=0, M=1, K=1),
                   dict(coarse=(8, 8, 16, 16), fine=(5, 5, 5, 5), levels=2, M=64, K=16)):
            refine_partition(ctx, ev, 0, dtype, stride, lam, **kw)          # warm: allocations
            runs.append(refine_partition(ctx, ev, 0, dtype, stride, lam, **kw))
        d, r = runs
        for res, acc in ((d, dense), (r, itr)):
            lv = res["levels"][-1]
            sd = lv["best_seed"]
            acc.append((lv["best_rss"], abs(float(np.linalg.norm(sd[3:])) - p_true), res["ms"],
                        sum(x["seeds"] for x in res["levels"])))
    ctx.close()

    def summ(a):
        a = np.array(a)
        return {"mean_best_rss": float(a[:, 0].mean()), "mean_abs_dp_MeV": float(a[:, 1].mean()),
                "rms_dp_MeV": float(np.sqrt((a[:, 1] ** 2).mean())), "mean_ms": float(a[:, 2].mean()),
                "seeds": int(a[0, 3])}
    wins = float(np.mean([b[0] <= a[0] for a, b in zip(dense, itr)]))
    return [{"study": "iterative", "events": n_events, "stride": stride, "lambda_mm": lam * 1e3,
             "dense_16x16x32x32": summ(dense), "iterative_2^14+2x16x5^4": summ(itr),
             "iterative_rss_le_dense": wins}]


class GaussNewton:
    """Gauss-Newton refinement of a few seeds of one turn partition (FP64, uniform axial field):
    each iteration is comet_scan_jacobian (smoothed RSS, normal equations) then comet_scan_gn_step,
    all on the device."""

    def __init__(self, ctx, ev, part: int, stride: int = 16, lam: float = 8e-4, tau: float = 1e-3,
                 K: int = 16):
        self.ctx, self.ev, self.tau, self.K = ctx, ev, tau, K
        spec = ev.partitions[part]
        self.spec = spec
        self.field = B.DeviceField.from_synth(synth.uniform_field(1.0))
        self.params = scan.params_for(spec, ev.n_steps[part], torch.float64, stride, lam)
        self.dev = scan.DeviceEvent.from_event(ev, torch.float64)
        W = max(self.dev.W, 1)
        f64 = dict(dtype=torch.float64, device="cuda")
        self.theta = torch.zeros((K, 4), **f64)
        self.work = torch.empty(K * W * B.JAC_WORK_PER_PAIR, **f64)
        self.srss = torch.empty(K, **f64)
        self.grad = torch.empty((K, 4), **f64)
        self.jtj = torch.empty((K, 16), **f64)
        self.jtr = torch.empty((K, 4), **f64)

    def evaluate(self, tau: Optional[float] = None):
        B.comet_scan_jacobian(self.ctx, self.field, self.params, self.theta, self.spec.vxy[0],
                              self.spec.vxy[1], self.spec.charge, self.dev.wires, self.dev.hit_offsets,
                              self.dev.drift, self.dev.mask, self.tau if tau is None else tau, self.work,
                              self.srss, self.grad, self.jtj, self.jtr, n_wires=self.dev.W)

    def run(self, iters: int = 10, mu: float = 1e-3):
        for _ in range(iters):
            self.evaluate()
            B.comet_scan_gn_step(self.ctx, self.theta, self.jtj, self.jtr, mu)
        self.evaluate()

    def _eval_at(self, theta, srss, grad, jtj, jtr, tau=None):
        B.comet_scan_jacobian(self.ctx, self.field, self.params, theta, self.spec.vxy[0],
                              self.spec.vxy[1], self.spec.charge, self.dev.wires, self.dev.hit_offsets,
                              self.dev.drift, self.dev.mask, self.tau if tau is None else tau, self.work,
                              srss, grad, jtj, jtr, n_wires=self.dev.W)

    def run_lm(self, iters: int = 10, mu0: float = 1e-3):
        """Levenberg-Marquardt: each iteration evaluates the trial seeds (one comet_scan_jacobian)
        and comet_scan_lm_step accepts a seed's trial only if its smoothed RSS is lower (the
        damping adapts per seed) and forms the next trial; theta ends at the accepted seeds."""
        if not hasattr(self, "t_theta"):
            f64 = dict(dtype=torch.float64, device="cuda")
            K = self.K
            self.t_theta = torch.empty((K, 4), **f64)
            self.t_srss = torch.empty(K, **f64)
            self.t_grad = torch.empty((K, 4), **f64)
            self.t_jtj = torch.empty((K, 16), **f64)
            self.t_jtr = torch.empty((K, 4), **f64)
            self.mu = torch.empty(K, **f64)
        self.mu.fill_(mu0)
        self.evaluate()
        B.comet_scan_lm_step(self.ctx, self.theta, self.srss, self.jtj, self.jtr, self.t_theta, None, None,
                             None, self.mu, first=True)
        for _ in range(iters):
            self._eval_at(self.t_theta, self.t_srss, self.t_grad, self.t_jtj, self.t_jtr)
            B.comet_scan_lm_step(self.ctx, self.theta, self.srss, self.jtj, self.jtr, self.t_theta,
                                 self.t_srss, self.t_jtj, self.t_jtr, self.mu)

    def hard_rss(self):
        """srss <- Eq. 1's capped RSS of the current seeds (the smooth cap at tau -> 0)."""
        self.evaluate(tau=1e-12)


def gn_study(n_events: int = 32, stride: int = 16, lam: float = 8e-4, iters: int = 10, K: int = 16,
             tau: float = 1e-3):
    """The dense 2^18 grid (FP32) against Gauss-Newton on the top K of a 2^14 grid (FP32 scan, then
    FP64 Gauss-Newton on the smoothed RSS; the seed of lowest capped RSS is kept): momentum error of
    the selected seed against the truth and warm GPU time.  Also the coarse grid's own best seed, and
    Levenberg-Marquardt with per-seed accept/reject (comet_scan_lm_step) from the same start."""
    ctx = B.Context(torch.cuda.current_device())
    dense, gn, coarse_only, lm = [], [], [], []
    for i in range(n_events):
        ev = synth.multi_turn_event(i)
        p_true = float(np.hypot(ev.pt, ev.pz))
        kw = dict(coarse=(16, 16, 32, 32), levels=0, M=1, K=1)
        refine_partition(ctx, ev, 0, torch.float32, stride, lam, **kw)
        d = refine_partition(ctx, ev, 0, torch.float32, stride, lam, **kw)
        sd = d["levels"][-1]["best_seed"]
        dense.append((abs(float(np.linalg.norm(sd[3:])) - p_true), d["ms"]))
        G = GaussNewton(ctx, ev, 0, stride, lam, tau=tau, K=K)
        res = None
        for rep in range(2):                                     # second run timed (warm)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            c = refine_partition(ctx, ev, 0, torch.float32, stride, lam, coarse=(8, 8, 16, 16),
                                 levels=0, M=64, K=1, keep_top=K)
            B.comet_scan_refine_refs(ctx, c["seeds"], c["idx"], [0.0] * 4, K, G.theta, c["nref"])
            th0 = G.theta[0].clone()
            G.run(iters)
            G.hard_rss()
            t1.record()
            t1.synchronize()
            res = (G.srss.cpu().numpy(), G.theta.cpu().numpy(), t0.elapsed_time(t1), th0.cpu().numpy())
        srss, theta, ms, th0 = res
        b = int(np.argmin(np.where(np.isfinite(srss), srss, np.inf)))
        gn.append((abs(float(np.hypot(theta[b, 2], theta[b, 3])) - p_true), ms))
        coarse_only.append((abs(float(np.hypot(th0[2], th0[3])) - p_true), 0.0))
        for rep in range(2):                                     # second run timed (warm)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            c = refine_partition(ctx, ev, 0, torch.float32, stride, lam, coarse=(8, 8, 16, 16),
                                 levels=0, M=64, K=1, keep_top=K)
            B.comet_scan_refine_refs(ctx, c["seeds"], c["idx"], [0.0] * 4, K, G.theta, c["nref"])
            G.run_lm(iters)
            G.hard_rss()
            t1.record()
            t1.synchronize()
            res = (G.srss.cpu().numpy(), G.theta.cpu().numpy(), t0.elapsed_time(t1))
        srss, theta, ms = res
        b = int(np.argmin(np.where(np.isfinite(srss), srss, np.inf)))
        lm.append((abs(float(np.hypot(theta[b, 2], theta[b, 3])) - p_true), ms))
    ctx.close()

    def summ(a):
        a = np.array(a)
        return {"mean_abs_dp_MeV": float(a[:, 0].mean()), "rms_dp_MeV": float(np.sqrt((a[:, 0] ** 2).mean())),
                "mean_ms": float(a[:, 1].mean())}
    return [{"study": "gauss-newton", "events": n_events, "stride": stride, "lambda_mm": lam * 1e3,
             "tau_mm": tau * 1e3, "iterations": iters, "K": K, "dense_16x16x32x32": summ(dense),
             "gn_top16_of_2^14": summ(gn), "lm_top16_of_2^14": summ(lm),
             "coarse_2^14_best": summ(coarse_only)}]


def generate_batch_events(n: int, workers: int = 0):
    """Events 0..n-1 of the batching workload (synth.batch_event), generated in a spawn process
    pool (the generator is NumPy only)."""
    import multiprocessing as mp
    import os
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1:
        return [synth.batch_event(i) for i in range(n)]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(synth.batch_event, range(n), chunksize=4)


def batch_study(n_events: int = 512, stride: int = 32, lam: float = 1e-2, tune_events: int = 128,
                dtype=torch.float32, max_total_seeds: int = 1 << 25):
    """Events/s and per-event latency of the batching workload (1-6 turns, 2^12-2^18 seeds per
    partition by turn count, uneven hit counts): the per-event path (one partition at a time, four
    launches each; and with each partition's recording beside the previous partition's DCA)
    against continuous batching (comet_scan_batch rounds replayed from a CUDA graph,
    configured by the autotuner on the first ``tune_events`` events)."""
    from . import batch as BT
    events = generate_batch_events(n_events)
    ctx = B.Context(torch.cuda.current_device())
    field = B.DeviceField.from_synth(synth.uniform_field(1.0))
    # per-event path
    S = max(sp.n_seeds for ev in events for sp in ev.partitions)
    n_rec = max(n // stride + 1 for ev in events for n in ev.n_steps)
    ws = scan.Workspace(S, n_rec, max(ev.n_hits for ev in events), dtype)
    devs = [scan.DeviceEvent.from_event(ev, dtype) for ev in events]
    for ev, dev in zip(events[:8], devs[:8]):
        scan.scan_event(ctx, field, ev, dev, ws, dtype, stride, lam)
    torch.cuda.synchronize()
    lat = []
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all0.record()
    for ev, dev in zip(events, devs):
        dev.mask.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        scan.scan_event(ctx, field, ev, dev, ws, dtype, stride, lam)
        b.record()
        lat.append((a, b))
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all1.record()
    torch.cuda.synchronize()
    seq_ms = t_all0.elapsed_time(t_all1)
    seq_lat = np.array([a.elapsed_time(b) for a, b in lat])
    del ws
    torch.cuda.empty_cache()
    # per-event path with each partition's recording beside the previous partition's DCA
    # (PipelinedScanner, the benchmark's driver): the same kernels, events back to back
    ps = scan.PipelinedScanner(ctx, field, S, n_rec, max(ev.n_hits for ev in events), dtype)
    params = [scan.event_params(ev, dtype, stride, lam) for ev in events]
    for i in range(8):
        devs[i].mask.zero_()
        ps.event(events[i], devs[i], params[i])
    torch.cuda.synchronize()
    lat = []
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all0.record()
    for ev, dev, prm in zip(events, devs, params):
        dev.mask.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ps.event(ev, dev, prm)
        b.record()
        lat.append((a, b))
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all1.record()
    torch.cuda.synchronize()
    pipe_ms = t_all0.elapsed_time(t_all1)
    pipe_lat = np.array([a.elapsed_time(b) for a, b in lat])
    ps.close()
    del ps, devs
    torch.cuda.empty_cache()
    # batched path
    sc = BT.BatchScanner(ctx, dtype, stride, lam, slots=256, max_total_seeds=max_total_seeds,
                         max_wires=max(512, max(ev.n_wires for ev in events)),
                         max_hits=max(2048, max(ev.n_hits for ev in events)))
    best, table = BT.autotune(sc, events[:tune_events], slots_options=(64, 128, 256), ctas_options=(0, 4),
                              graph_options=(True, False), solo_options=(None, 1 << 16, 1 << 17),
                              lanes_options=(1, 2, 3, 4), chunk_options=(0, 16, 64),
                              item_options=(0, 4, 16))
    pinned = sc.pin(events)
    sc.run(events[:tune_events], pinned=pinned[:tune_events])
    r = sc.run(events, pinned=pinned)
    sc.close_lanes()
    # two scanners (two contexts and streams) with the tuned configuration, rounds interleaved
    half = max(1, max_total_seeds // 2)
    ctx2 = B.Context(torch.cuda.current_device())
    del sc
    torch.cuda.empty_cache()
    pair = [BT.BatchScanner(c, dtype, stride, lam, slots=best["slots"], max_total_seeds=half,
                            max_wires=max(512, max(ev.n_wires for ev in events)),
                            max_hits=max(2048, max(ev.n_hits for ev in events)),
                            graph=best["graph"], dca_ctas_per_sm=best["dca_ctas_per_sm"],
                            solo_min_seeds=best["solo_min_seeds"], solo_lanes=best["solo_lanes"],
                            chunk_wires=best["chunk_wires"], item_groups=best["item_groups"])
            for c in (ctx, ctx2)]
    BT.run_interleaved(pair, events[:tune_events])
    r2 = BT.run_interleaved(pair, events)
    for sc2 in pair:
        sc2.close_lanes()
    del pair
    ctx2.close()
    wires = np.array([ev.n_wires for ev in events])
    turns = np.bincount([len(ev.partitions) for ev in events], minlength=7)[1:]
    ctx.close()
    pct = lambda x: {"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99))}
    return [{"study": "batch", "events": n_events, "stride": stride, "lambda_mm": lam * 1e3,
             "turns_1_to_6": turns.tolist(), "wires_min_median_max": [int(wires.min()), int(np.median(wires)),
                                                                      int(wires.max())],
             "per_event_path": {"events_per_s": n_events / (seq_ms * 1e-3), "latency_ms": pct(seq_lat)},
             "per_event_pipelined": {"events_per_s": n_events / (pipe_ms * 1e-3), "latency_ms": pct(pipe_lat)},
             "batched": {"events_per_s": n_events / (r["gpu_ms"] * 1e-3), "latency_ms": pct(r["latency_ms"]),
                         "rounds": r["rounds"], "host_wall_ms": r["wall_ms"], "gpu_ms": r["gpu_ms"],
                         "config": best},
             "batched_two_streams": {"events_per_s": n_events / (r2["gpu_ms"] * 1e-3),
                                     "latency_ms": pct(r2["latency_ms"]), "rounds": r2["rounds"]},
             "autotune": table}]


def table_field_study(n_events: int = 8, stride: int = 16, lam: float = 1e-2, dtype=torch.float32):
    """Seed x hit DCA evaluations/s on the non-uniform-field workload (DIO-shaped momenta 50-105
    MeV/c, the tabulated solenoid model, 2^18 seeds per partition): every RK4 step of the track
    recording and of the refinement evaluates the trilinear table.  The same events scanned in the
    uniform 1 T field (the closed-form axial map) are timed beside them."""
    fld = synth.table_field()
    events = [synth.table_field_event(i, fld) for i in range(n_events)]
    ctx = B.Context(torch.cuda.current_device())
    out = {"study": "table-field", "events": n_events, "stride": stride, "lambda_mm": lam * 1e3,
           "momenta_MeV": [round(float(np.hypot(ev.pt, ev.pz)), 1) for ev in events]}
    for name, field, il in (("table", fld, False), ("table_interleaved", fld, True),
                            ("uniform", synth.uniform_field(1.0), False)):
        dfield = B.DeviceField.from_synth(field, interleaved=il)
        S = max(sp.n_seeds for ev in events for sp in ev.partitions)
        n_rec = max(n // stride + 1 for ev in events for n in ev.n_steps)
        ws = scan.Workspace(S, n_rec, max(ev.n_hits for ev in events), dtype)
        devs = [scan.DeviceEvent.from_event(ev, dtype) for ev in events]
        scan.scan_event(ctx, dfield, events[0], devs[0], ws, dtype, stride, lam)
        evals = 0
        timer = scan.KernelTimer()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        classes = []
        for ev, dev in zip(events, devs):
            dev.mask.zero_()
            cl = []
            for spec, p in zip(ev.partitions, scan.event_params(ev, dtype, stride, lam)):
                scan.scan_partition(ctx, dfield, p, spec, dev, ws, timer=timer)
                cl.append(ws.hit_class[: max(ev.n_hits, 1)].clone())
            classes.append(cl)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        for ev, cl in zip(events, classes):
            masked = np.zeros(ev.n_hits, bool)
            for spec, c in zip(ev.partitions, cl):
                evals += spec.n_seeds * int((~masked).sum())
                masked |= c.cpu().numpy()[: ev.n_hits].astype(bool)
        out[name] = {"evals_per_s": evals / (ms * 1e-3), "ms_per_event": ms / n_events,
                     "kernel_ms": {k: round(v[0], 3) for k, v in timer.totals().items()}}
        del ws, devs
        torch.cuda.empty_cache()
    ctx.close()
    return [out]


def single_event_study(reps: int = 50, stride: int = 16, lam: float = 1e-2):
    """The single-event configuration (p = 104 MeV/c at 80 degrees, 2 turn partitions of 8^4 seeds,
    131 hits on 106 wires) in FP64 and in FP32: per-kernel GPU time per event, seed x hit
    evaluations/s, and the DCA kernel's algorithmic flop rate (201 flops per seed x wire with an
    unmasked hit + 8 per seed x unmasked hit) against the nominal FP64 rate of this part
    (1.25 TFLOP/s, not measured here) and the derived FP32 peak (80.5 TFLOP/s).  At 4096 seeds per
    partition the launches are latency-bound: the fractions say how little of the part such a
    small scan uses, not how fast the kernels are."""
    ev = synth.single_event_fp64()
    out = {"study": "single-event", "reps": reps, "stride": stride, "lambda_mm": lam * 1e3,
           "seeds_per_partition": ev.partitions[0].n_seeds, "partitions": len(ev.partitions),
           "hits": ev.n_hits, "wires": ev.n_wires}
    offs = np.asarray(ev.hit_offsets)
    for name, dtype, peak in (("fp64", torch.float64, 1.25), ("fp32", torch.float32, 80.54784)):
        ctx, field, ws = _setup([ev], dtype, stride)
        dev = scan.DeviceEvent.from_event(ev, dtype)
        params = scan.event_params(ev, dtype, stride, lam)
        classes = [torch.zeros(max(ev.n_hits, 1), dtype=torch.uint8, device="cuda") for _ in ev.partitions]

        def run(timer=None):
            dev.mask.zero_()
            for p, (spec, bp) in enumerate(zip(ev.partitions, params)):
                scan.scan_partition(ctx, field, bp, spec, dev, ws, hit_class=classes[p], timer=timer)

        for _ in range(3):
            run()
        # whole events: one event pair around `reps` back-to-back events
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        # per kernel: events between the steps (they include the host's launch gaps)
        timer = scan.KernelTimer()
        for _ in range(reps):
            run(timer)
        torch.cuda.synchronize()
        kt = {k: v[0] / reps for k, v in timer.totals().items()}
        masked = np.zeros(ev.n_hits, bool)
        hits = wires = 0
        for spec, cls in zip(ev.partitions, classes):
            live = ~masked
            # unmasked hits per wire (wires without hits count 0)
            csum = np.concatenate([[0], np.cumsum(live.astype(np.int64))])
            per_wire = csum[offs[1:]] - csum[offs[:-1]]
            hits += spec.n_seeds * int(live.sum())
            wires += spec.n_seeds * int((per_wire > 0).sum())
            masked |= cls[: ev.n_hits].cpu().numpy().astype(bool)
        flops = 201 * wires + 8 * hits
        out[name] = {"ms_per_event": ms, "sum_kernel_ms": sum(kt.values()),
                     "kernel_ms": {k: round(v, 4) for k, v in kt.items()},
                     "evals_per_s": hits / (ms * 1e-3),
                     "dca_tflops": flops / (kt["dca"] * 1e-3) / 1e12,
                     "dca_frac": flops / (kt["dca"] * 1e-3) / 1e12 / peak,
                     "peak_tflops": peak, "peak_source": "nominal" if name == "fp64" else "derived"}
        ctx.close()
    return [out]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["lambda-sweep", "backward", "iterative", "gauss-newton", "batch",
                                      "table-field", "single-event"])
    ap.add_argument("--reps", type=int, default=50, help="timed repetitions (single-event)")
    ap.add_argument("--events", type=int, default=32)
    ap.add_argument("--stride", type=int, default=16)
    ap.add_argument("--lambda-mm", type=float, default=10.0, help="cutoff (backward, iterative, gn)")
    ap.add_argument("--tau-mm", type=float, default=1.0, help="smoothing width of the gn study")
    args = ap.parse_args(argv)
    if args.study == "lambda-sweep":
        rows = lambda_sweep(args.events, stride=args.stride)
    elif args.study == "iterative":
        rows = iterative_study(args.events, args.stride, args.lambda_mm * 1e-3)
    elif args.study == "single-event":
        rows = single_event_study(args.reps, args.stride, args.lambda_mm * 1e-3)
    elif args.study == "table-field":
        rows = table_field_study(args.events, args.stride, args.lambda_mm * 1e-3)
    elif args.study == "batch":
        rows = batch_study(args.events, args.stride, args.lambda_mm * 1e-3)
    elif args.study == "gauss-newton":
        rows = gn_study(args.events, args.stride, args.lambda_mm * 1e-3, tau=args.tau_mm * 1e-3)
    else:
        rows = backward_study(args.events, args.stride, args.lambda_mm * 1e-3)
    for r in rows:
        print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
