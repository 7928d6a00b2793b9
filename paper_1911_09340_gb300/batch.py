"""Many events at once: continuous batching of the scan over event slots (comet_scan_batch).

Each of ``slots`` slots holds one event for its lifetime: its wires, hits and hit mask stay on the
device while its turn partitions are scanned one per round, in order (hits classified at one
partition are masked for the next, Sec. 3.1).  A round is ONE comet_scan_batch: the current
partition of every active slot in single batched launches.  When an event's last partition is
done its slot takes the next event of the queue.  The per-round scratch (seeds, track points,
search bounds, RSS) is bump-allocated from arenas sized by the caps; a round that would exceed the
seed or wire budget leaves the remaining slots waiting for the next round.

With ``graph=True`` the work comet_scan_batch enqueues is captured once in a CUDA graph and every
round replays it after comet_scan_batch_update has packed the round's descriptors (grid sizes
depend on the caps only).

Size-aware rounds (``solo_min_seeds``): a partition of that many seeds or more fills the GPU by
itself, so it runs through the single-event calls (lattice, propagate, dca with the selection,
classify on the slot's resident buffers) on one of ``solo_lanes`` lanes (each its own context,
stream and workspace), while the round's smaller partitions run as one batch on the scanner's
stream -- the big partitions keep the single-event kernels' efficiency, the small ones share
launches, and each fills the others' kernel tails.  All streams join at the end of a round.

The host work per round is descriptor packing; every step of the scan runs in the library's
kernels.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
from collections import deque
from typing import Dict, List, Optional

import numpy as np
import torch

from . import binding as B
from . import scan, synth


def _pad4(n: int) -> int:
    return max(4, (n + 3) // 4 * 4)


@dataclasses.dataclass
class EventResult:
    best_idx: List[int]
    best_rss: List[float]
    hit_class: List[np.ndarray]
    start_round: int = -1
    end_round: int = -1


class BatchScanner:
    def __init__(self, ctx: B.Context, dtype=torch.float32, stride: int = 16, lam: float = 1e-2,
                 slots: int = 128, max_seeds: int = 1 << 18, max_total_seeds: int = 1 << 24,
                 max_wires: int = 512, max_hits: int = 2048, max_n_steps: int = 2400,
                 graph: bool = True, field: Optional[synth.Field] = None, dca_ctas_per_sm: int = 0,
                 solo_min_seeds: Optional[int] = None, solo_lanes: int = 1, chunk_wires: int = 0,
                 item_groups: int = 0):
        self.ctx, self.dtype, self.stride, self.lam = ctx, dtype, stride, lam
        self.slots = self.slots_alloc = slots
        self.max_hits = max_hits
        self.field = B.DeviceField.from_synth(field or synth.uniform_field(1.0))
        self.params = B.ScanParams(n_steps=max_n_steps, stride=stride, lam=lam,
                                   tol=1e-12 if dtype == torch.float64 else 1e-6, max_iter=16)
        self.max_seeds, self.max_total_seeds, self.max_wires = max_seeds, max_total_seeds, max_wires
        self.dca_ctas_per_sm = dca_ctas_per_sm
        self.item_groups = item_groups        # 32-seed groups per batched DCA item (0: automatic)
        self.chunk_wires = chunk_wires        # wires per chunk of the DCA's sums (0: automatic)
        ctx.set_dca_chunk_wires(chunk_wires)
        self.caps = self._caps(slots, dca_ctas_per_sm)
        self.n_rec_max = max_n_steps // stride + 1
        dev = dict(device="cuda")
        es = torch.tensor([], dtype=dtype).element_size()
        self.es = es
        # per-round arenas
        T = max_total_seeds
        self.a_seeds = torch.empty(6 * T, dtype=dtype, **dev)
        self.a_charge = torch.empty(T, dtype=torch.int8, **dev)
        self.a_points = torch.empty(6 * self.n_rec_max * T, dtype=dtype, **dev)
        self.a_nvalid = torch.empty(T, dtype=torch.int32, **dev)
        self.a_bounds = torch.empty(((T + 31) // 32 + slots) * B.BOUNDS_PER_GROUP * 4, dtype=torch.float32, **dev)
        self.a_rss = torch.empty(T, dtype=dtype, **dev)
        self.a_nin = torch.empty(T, dtype=torch.int32, **dev)
        # per-slot resident buffers
        self.ldw = _pad4(max_wires)
        self.s_wires = torch.zeros((slots, 6, self.ldw), dtype=dtype, **dev)
        self.s_offs = torch.zeros((slots, max_wires + 1), dtype=torch.int32, **dev)
        self.s_drift = torch.zeros((slots, max_hits), dtype=dtype, **dev)
        self.s_mask = torch.zeros((slots, max_hits), dtype=torch.uint8, **dev)
        self.s_class = torch.zeros((slots, max_hits), dtype=torch.uint8, **dev)
        self.s_best = torch.zeros(slots, dtype=torch.int64, **dev)
        self.s_best_rss = torch.zeros(slots, dtype=dtype, **dev)
        self.s_unconv = torch.zeros(slots, dtype=torch.int32, **dev)
        self.desc = (B.BatchEvent * slots)()
        self.graphs = {}                 # captured rounds, per caps
        self.use_graph = graph
        self.stream = torch.cuda.Stream()
        # partitions of at least this many seeds run alone through the single-event calls, spread
        # round-robin over `solo_lanes` lanes (a context, a stream and a workspace each: one
        # context's DCA calls must not overlap on the GPU, those of different contexts may)
        self.solo_min_seeds = solo_min_seeds
        self.solo_lanes = solo_lanes
        self._lanes = []                 # [(context, stream, workspace)], made on first use
        self.solo_params = {}

    def _caps(self, slots: int, dca_ctas_per_sm: int) -> B.BatchCaps:
        return B.BatchCaps(slots, self.max_seeds, self.max_total_seeds, self.max_wires,
                           slots * self.max_wires, dca_ctas_per_sm, self.item_groups)

    def configure(self, slots: Optional[int] = None, dca_ctas_per_sm: Optional[int] = None,
                  graph: Optional[bool] = None, solo_min_seeds=-1, solo_lanes: Optional[int] = None,
                  chunk_wires: Optional[int] = None, item_groups: Optional[int] = None):
        """Events in flight (at most the slots allocated), DCA CTAs per SM, graph use, the solo
        threshold (None: every partition batched), the number of solo lanes, the DCA's wires per
        chunk and the batched DCA's seed groups per item of the next runs (the knobs the autotuner
        turns; 0 = automatic for the last two)."""
        if solo_min_seeds != -1:
            self.solo_min_seeds = solo_min_seeds
        if solo_lanes is not None:
            self.solo_lanes = max(1, int(solo_lanes))
        if chunk_wires is not None:
            self.chunk_wires = int(chunk_wires)
            self.ctx.set_dca_chunk_wires(self.chunk_wires)
            for c, _, _ in self._lanes[1:]:
                c.set_dca_chunk_wires(self.chunk_wires)
        if item_groups is not None:
            self.item_groups = int(item_groups)
        if slots is not None:
            if slots > self.slots_alloc:
                raise ValueError("more slots than allocated")
            self.slots = slots
        if dca_ctas_per_sm is not None:
            self.dca_ctas_per_sm = dca_ctas_per_sm
        if graph is not None:
            self.use_graph = graph
        caps = self._caps(self.slots, self.dca_ctas_per_sm)
        if ((caps.max_events, caps.dca_ctas_per_sm, caps.dca_item_groups) !=
                (self.caps.max_events, self.caps.dca_ctas_per_sm, self.caps.dca_item_groups)):
            # the next update reallocates the context's staging buffers that captured graphs copy
            # from: a graph captured before must never be replayed again
            self.graphs.clear()
        self.caps = caps

    # ---- slots -----------------------------------------------------------------------------------
    def pin(self, events):
        """Pinned host copies of the events' wires, offsets and drifts, so that loading an event
        into a slot is an asynchronous copy (the host packs the next round meanwhile)."""
        out = []
        for ev in events:
            W, H = ev.n_wires, ev.n_hits
            if W > self.caps.max_wires or H > self.max_hits:
                raise ValueError(f"event with W={W}, H={H} exceeds the scanner's caps")
            w = torch.zeros((6, self.ldw), dtype=self.dtype)
            w[:, :W] = torch.as_tensor(ev.wires, dtype=self.dtype)
            out.append((w.pin_memory(), torch.as_tensor(np.asarray(ev.hit_offsets, np.int32)).pin_memory(),
                        torch.as_tensor(ev.drift, dtype=self.dtype).pin_memory()))
        return out

    def _load(self, slot: int, ev, pinned):
        W, H = ev.n_wires, ev.n_hits
        w, o, d = pinned
        self.s_wires[slot].copy_(w, non_blocking=True)
        self.s_offs[slot, : W + 1].copy_(o, non_blocking=True)
        if H:
            self.s_drift[slot, :H].copy_(d, non_blocking=True)
        self.s_mask[slot].zero_()

    def _fill(self, slot: int, ev, part: int, o_s: int, o_b: int):
        d = self.desc[slot]
        spec = ev.partitions[part]
        S = spec.n_seeds
        n = ev.n_steps[part]
        d.active = 1
        d.lattice = B.lattice_struct(spec)
        d.n_steps = n
        es = self.es
        d.seeds = self.a_seeds.data_ptr() + 6 * o_s * es
        d.charge = self.a_charge.data_ptr() + o_s
        d.points = self.a_points.data_ptr() + 6 * self.n_rec_max * o_s * es
        d.n_valid = self.a_nvalid.data_ptr() + 4 * o_s
        d.bounds = self.a_bounds.data_ptr() + o_b * B.BOUNDS_PER_GROUP * 16
        d.wires = self.s_wires[slot].data_ptr()
        d.W = ev.n_wires
        d.ldw = self.ldw
        d.hit_offsets = self.s_offs[slot].data_ptr()
        d.drift = self.s_drift[slot].data_ptr()
        d.hit_mask = self.s_mask[slot].data_ptr()
        d.rss = self.a_rss.data_ptr() + o_s * es
        d.n_in = self.a_nin.data_ptr() + 4 * o_s
        d.best_idx = self.s_best[slot:].data_ptr()
        d.best_rss = self.s_best_rss[slot:].data_ptr()
        d.hit_class = self.s_class[slot].data_ptr()
        d.n_unconverged = self.s_unconv[slot:].data_ptr()
        return S

    def _lane(self, k: int):
        while len(self._lanes) <= k:
            c = self.ctx if not self._lanes else B.Context(self.ctx.device)
            c.set_dca_chunk_wires(self.chunk_wires)
            c.set_record_blocks(self.ctx.record_blocks)
            self._lanes.append((c, torch.cuda.Stream(),
                                scan.Workspace(self.max_seeds, self.n_rec_max, 1, self.dtype)))
        return self._lanes[k]

    def close_lanes(self):
        """Releases the extra contexts of the solo lanes (the first lane uses the scanner's)."""
        torch.cuda.synchronize()
        for c, _, _ in self._lanes[1:]:
            c.close()
        self._lanes = []

    def _solo(self, lane, slot: int, ev, part: int):
        """One partition of the event in ``slot`` through the single-event calls on a solo lane
        (context, stream, workspace), reading and updating the slot's resident hits and mask and
        writing its outputs."""
        ctx, st, ws = lane
        spec = ev.partitions[part]
        S = spec.n_seeds
        n = ev.n_steps[part]
        key = n
        bp = self.solo_params.get(key)
        if bp is None:
            bp = B.ScanParams(n_steps=n, stride=self.stride, lam=self.lam, tol=self.params.tol,
                              max_iter=self.params.max_iter)
            self.solo_params[key] = bp
        seeds, charge, pts, nv, rss, n_in = ws.views(S, bp.n_rec)
        W, H = ev.n_wires, ev.n_hits
        wires = self.s_wires[slot]
        offs = self.s_offs[slot, : W + 1]
        drift = self.s_drift[slot, : max(H, 1)]
        mask = self.s_mask[slot, : max(H, 1)]
        bounds = ws.bounds[: (S + 31) // 32]
        B.comet_scan_lattice(ctx, spec, seeds, charge, stream=st)
        B.comet_scan_propagate(ctx, self.field, bp, seeds, charge, pts, nv, bounds=bounds, stream=st)
        B.comet_scan_dca(ctx, self.field, bp, pts, nv, charge, wires, offs, drift, mask, rss, n_in,
                         n_unconverged=self.s_unconv[slot:slot + 1], n_wires=W, bounds=bounds, stream=st,
                         best_idx=self.s_best[slot:slot + 1], best_rss=self.s_best_rss[slot:slot + 1])
        if W > 0:
            B.comet_scan_classify(ctx, self.field, bp, pts, nv, charge, self.s_best[slot:slot + 1],
                                  wires, offs, drift, mask, self.s_class[slot, : max(H, 1)],
                                  update_mask=True, n_wires=W, stream=st)

    # ---- the run -----------------------------------------------------------------------------------
    def run(self, events, collect: bool = False, pinned=None) -> Dict:
        """Scans every partition of every event.  Returns per-event results (when ``collect``: best
        seed, its RSS and the hit classes of each partition), per-event latency in ms (from the end
        of the round before its first partition to the end of its last) and the total GPU time.
        ``pinned`` = self.pin(events), made once (else made here, untimed)."""
        return run_interleaved([self], events, collect, [pinned] if pinned is not None else None)

    def rounds(self, events, pinned, results, collect: bool):
        """Generator: packs and launches one round per step (on this scanner's stream) and yields
        the CUDA event recorded after it; fills ``results`` (start/end rounds, and the outputs when
        ``collect``)."""
        queue = deque(range(len(events)))
        state = [None] * self.slots          # (event index, next partition)
        rnd = 0
        start = 0
        while queue or any(s is not None for s in state):
            with torch.cuda.stream(self.stream):
                for slot in range(self.slots):
                    if state[slot] is None and queue:
                        i = queue.popleft()
                        self._load(slot, events[i], pinned[i])
                        state[slot] = (i, 0)
                        results[i].start_round = rnd
                o_s = o_b = w_tot = 0
                members, solos = [], []
                solo_min = self.solo_min_seeds
                for k in range(self.slots):
                    slot = (start + k) % self.slots
                    st = state[slot]
                    self.desc[slot].active = 0
                    if st is None:
                        continue
                    ev = events[st[0]]
                    S = ev.partitions[st[1]].n_seeds
                    if solo_min is not None and S >= solo_min:
                        solos.append(slot)
                        continue
                    if o_s + S > self.caps.max_total_seeds or w_tot + ev.n_wires > self.caps.max_total_wires:
                        continue                       # waits for the next round
                    self._fill(slot, ev, st[1], o_s, o_b)
                    o_s += S
                    o_b += (S + 31) // 32
                    w_tot += ev.n_wires
                    members.append(slot)
                start = (start + 1) % self.slots
                lanes = [self._lane(k) for k in range(min(self.solo_lanes, len(solos)))]
                if solos:
                    # the solo lanes start after this round's loads and the previous round
                    loaded = torch.cuda.Event()
                    loaded.record(self.stream)
                    for _, st_l, _ in lanes:
                        st_l.wait_event(loaded)
                    for n_s, slot in enumerate(solos):
                        i, p = state[slot]
                        self._solo(lanes[n_s % len(lanes)], slot, events[i], p)
                if members:
                    self._launch()
                for _, st_l, _ in lanes:
                    done = torch.cuda.Event()
                    done.record(st_l)
                    self.stream.wait_event(done)
                members += solos
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                if collect:
                    self.stream.synchronize()
                    best = self.s_best.cpu().numpy()
                    best_rss = self.s_best_rss.double().cpu().numpy()
                    cls = self.s_class.cpu().numpy()
            for slot in members:
                i, p = state[slot]
                if collect:
                    ev = events[i]
                    results[i].best_idx.append(int(best[slot]))
                    results[i].best_rss.append(float(best_rss[slot]))
                    results[i].hit_class.append(cls[slot, : ev.n_hits].copy())
                if p + 1 == len(events[i].partitions):
                    results[i].end_round = rnd
                    state[slot] = None
                else:
                    state[slot] = (i, p + 1)
            rnd += 1
            yield e

    def _launch(self):
        B.comet_scan_batch_update(self.ctx, self.dtype, self.field, self.params, self.caps, self.desc,
                                  self.slots)
        if not self.use_graph:
            B.comet_scan_batch(self.ctx, self.dtype, self.field, self.params, self.caps,
                               stream=self.stream)
            return
        key = (self.caps.max_events, self.caps.dca_ctas_per_sm,
               self.caps.dca_item_groups)                         # at most one entry (see configure)
        g = self.graphs.get(key)
        if g is None:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                B.comet_scan_batch(self.ctx, self.dtype, self.field, self.params, self.caps,
                                   stream=torch.cuda.current_stream())
            self.graphs[key] = g
        g.replay()


def run_interleaved(scanners, events, collect: bool = False, pinned=None) -> Dict:
    """Scans ``events`` with one or more scanners (each with its own context and stream): event i
    goes to scanner i mod n, and the scanners' rounds are launched alternately, so that the rounds
    of different scanners overlap on the GPU (one scanner's kernel tails are filled by another's
    work).  Same results as one scanner; latency and GPU time as in BatchScanner.run."""
    import time
    n = len(scanners)
    parts = [list(range(k, len(events), n)) for k in range(n)]
    sub = [[events[i] for i in part] for part in parts]
    pins = pinned if pinned is not None else [sc.pin(ev) for sc, ev in zip(scanners, sub)]
    res = [[EventResult([], [], []) for _ in ev] for ev in sub]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    t0 = torch.cuda.Event(enable_timing=True)
    t0.record()
    gens = [sc.rounds(ev, pn, r, collect) for sc, ev, pn, r in zip(scanners, sub, pins, res)]
    marks = [[] for _ in scanners]
    live = list(range(n))
    while live:
        for k in list(live):
            try:
                marks[k].append(next(gens[k]))
            except StopIteration:
                live.remove(k)
    torch.cuda.synchronize()
    wall_ms = (time.perf_counter() - w0) * 1e3
    results = [None] * len(events)
    lat = np.zeros(len(events))
    gpu_ms = 0.0
    rounds = 0
    for k in range(n):
        ms = [t0.elapsed_time(m) for m in marks[k]]
        rounds = max(rounds, len(ms))
        if ms:
            gpu_ms = max(gpu_ms, ms[-1])
        for j, i in enumerate(parts[k]):
            r = res[k][j]
            results[i] = r
            begin = 0.0 if r.start_round <= 0 else ms[r.start_round - 1]
            lat[i] = ms[r.end_round] - begin
    return {"results": results, "latency_ms": lat, "gpu_ms": gpu_ms, "rounds": rounds, "wall_ms": wall_ms}


def autotune(scanner: BatchScanner, events, slots_options=(32, 64, 128, 256), ctas_options=(0, 4, 2),
             graph_options=(True, False), solo_options=(None,), lanes_options=(1,),
             chunk_options=(0,), item_options=(0,)):
    """Measures events/s of each (events in flight, DCA CTAs per SM, CUDA graph, solo threshold,
    solo lanes) on ``events`` (a sample of the workload; one warm run and one timed run each), then
    from the best of those each (wires per chunk, seed groups per batched DCA item), and leaves the
    scanner configured with the fastest.  Returns (best, table)."""
    table = []
    pinned = scanner.pin(events)
    for solo in solo_options:
        for nl in (lanes_options if solo is not None else (1,)):
            for g in graph_options:
                for sl in slots_options:
                    if sl > scanner.slots_alloc:
                        continue
                    for c in ctas_options:
                        scanner.configure(slots=sl, dca_ctas_per_sm=c, graph=g, solo_min_seeds=solo,
                                          solo_lanes=nl)
                        scanner.run(events, pinned=pinned)
                        r = scanner.run(events, pinned=pinned)
                        table.append({"slots": sl, "dca_ctas_per_sm": c, "graph": g,
                                      "solo_min_seeds": solo, "solo_lanes": nl,
                                      "chunk_wires": scanner.chunk_wires,
                                      "item_groups": scanner.item_groups,
                                      "events_per_s": len(events) / (r["gpu_ms"] * 1e-3),
                                      "gpu_ms": r["gpu_ms"]})
    best = max(table, key=lambda t: t["events_per_s"])
    scanner.configure(slots=best["slots"], dca_ctas_per_sm=best["dca_ctas_per_sm"], graph=best["graph"],
                      solo_min_seeds=best["solo_min_seeds"], solo_lanes=best["solo_lanes"])
    # second stage, from the best of the first: the DCA's wires per chunk (the work item's hit tile)
    # and the batched DCA's 32-seed groups per CTA item (its seeds per block); 0 = automatic
    for cw in chunk_options:
        for ig in item_options:
            if (cw, ig) == (0, 0):
                continue
            scanner.configure(chunk_wires=cw, item_groups=ig)
            scanner.run(events, pinned=pinned)
            r = scanner.run(events, pinned=pinned)
            row = dict(best, chunk_wires=cw, item_groups=ig,
                       events_per_s=len(events) / (r["gpu_ms"] * 1e-3), gpu_ms=r["gpu_ms"])
            table.append(row)
    best = max(table, key=lambda t: t["events_per_s"])
    scanner.configure(chunk_wires=best.get("chunk_wires", 0), item_groups=best.get("item_groups", 0))
    return best, table
