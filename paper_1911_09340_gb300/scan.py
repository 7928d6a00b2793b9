"""Event-level driver of the seed scan on one GPU.

An event's turn partitions are scanned in order (Sec. 3.1: a *stage* per turn; hits classified at
one stage are excluded from the next).  For each partition the five C-ABI calls run back to back on
the current stream with no host synchronisation:

    lattice -> propagate -> dca -> select -> classify (mask update)

Everything runs in the library's kernels; torch only provides device memory and the stream.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np
import torch

from . import binding as B

KAPPA = 299.792458


def _pad4(n: int) -> int:
    return max(4, (n + 3) // 4 * 4)


@dataclasses.dataclass
class DeviceEvent:
    """An event's hits on the device.  ``wires`` is [6][ldw] (ldw padded to a multiple of 4 so that
    every row starts on a 16-byte boundary for the bulk-copy engine)."""
    wires: torch.Tensor
    hit_offsets: torch.Tensor
    drift: torch.Tensor
    mask: torch.Tensor
    W: int
    H: int

    @classmethod
    def from_host(cls, wires: np.ndarray, hit_offsets: np.ndarray, drift: np.ndarray,
                  dtype=torch.float32, device="cuda", non_blocking: bool = False):
        W = int(wires.shape[1])
        H = int(drift.shape[0])
        w = torch.zeros((6, _pad4(W)), dtype=dtype, device=device)
        w[:, :W] = torch.as_tensor(np.asarray(wires), dtype=dtype).to(device, non_blocking=non_blocking)
        return cls(w, torch.as_tensor(np.asarray(hit_offsets, np.int32)).to(device),
                   torch.as_tensor(np.asarray(drift)).to(device=device, dtype=dtype),
                   torch.zeros(max(H, 1), dtype=torch.uint8, device=device), W, H)

    @classmethod
    def from_event(cls, ev, dtype=torch.float32, device="cuda"):
        return cls.from_host(ev.wires, ev.hit_offsets, ev.drift, dtype, device)


class Workspace:
    """Device buffers of one partition scan, sized for up to S seeds and n_rec recorded states."""

    def __init__(self, S: int, n_rec: int, H: int, dtype=torch.float32, k: int = 1,
                 device="cuda"):
        self.S, self.n_rec, self.dtype, self.k = S, n_rec, dtype, k
        self.seeds = torch.empty((6, S), dtype=dtype, device=device)
        self.charge = torch.empty(S, dtype=torch.int8, device=device)
        self.points = torch.empty((6, n_rec, S), dtype=dtype, device=device)
        self.n_valid = torch.empty(S, dtype=torch.int32, device=device)
        self.bounds = torch.empty(B.bounds_shape(S), dtype=torch.float32, device=device)
        self.rss = torch.empty(S, dtype=dtype, device=device)
        self.n_in = torch.empty(S, dtype=torch.int32, device=device)
        self.idx = torch.empty(k, dtype=torch.int64, device=device)
        self.best = torch.empty(k, dtype=dtype, device=device)
        self.hit_class = torch.empty(max(H, 1), dtype=torch.uint8, device=device)
        self.n_unconv = torch.zeros(1, dtype=torch.int32, device=device)

    def fits(self, S: int, n_rec: int, H: int) -> bool:
        return S <= self.S and n_rec <= self.n_rec and H <= self.hit_class.numel()

    def views(self, S: int, n_rec: int):
        """Contiguous views sized exactly for (S, n_rec)."""
        pts = self.points.view(-1)[: 6 * n_rec * S].view(6, n_rec, S)
        return (self.seeds.view(-1)[: 6 * S].view(6, S), self.charge[:S], pts, self.n_valid[:S],
                self.rss[:S], self.n_in[:S])


def params_for(spec, n_steps: int, dtype=torch.float32, stride: int = 1, lam: float = 1e-2,
               h: float = 1e-3) -> B.ScanParams:
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    return B.ScanParams(h=h, n_steps=n_steps, stride=stride, lam=lam, tol=tol, max_iter=16)


def scan_partition(ctx: B.Context, field: B.DeviceField, params: B.ScanParams, spec,
                   ev: DeviceEvent, ws: Workspace, k: int = 1, update_mask: bool = True,
                   want_dca: Optional[torch.Tensor] = None, dca_wire: Optional[torch.Tensor] = None,
                   hit_class: Optional[torch.Tensor] = None, timer=None,
                   best_idx: Optional[torch.Tensor] = None, best_rss: Optional[torch.Tensor] = None):
    """One turn partition: lattice -> propagate -> dca (with the selection when k = 1, else a
    select launch) -> classify.  Results stay on the device in ``ws`` (idx, best, rss, n_in,
    hit_class) and ``ev.mask`` (updated in place); with k = 1, ``best_idx`` / ``best_rss`` ([1]
    device tensors) take the selected seed and its RSS instead of ws.idx / ws.best."""
    S = spec.n_seeds
    seeds, charge, pts, nv, rss, n_in = ws.views(S, params.n_rec)
    mark = timer.mark if timer is not None else (lambda name: None)
    mark("lattice")
    B.comet_scan_lattice(ctx, spec, seeds, charge)
    mark("propagate")
    bounds = ws.bounds[: (S + 31) // 32]
    B.comet_scan_propagate(ctx, field, params, seeds, charge, pts, nv, bounds=bounds)
    mark("dca")
    # k = 1: the seed of lowest RSS is selected inside the DCA launch; top-k takes comet_scan_select
    fused = k == 1
    bi = (ws.idx[:1] if best_idx is None else best_idx) if fused else ws.idx
    br = (ws.best[:1] if best_rss is None else best_rss) if fused else None
    B.comet_scan_dca(ctx, field, params, pts, nv, charge, ev.wires, ev.hit_offsets, ev.drift,
                     ev.mask, rss, n_in, dca_out=want_dca, n_unconverged=ws.n_unconv, n_wires=ev.W,
                     bounds=bounds, best_idx=bi if fused else None, best_rss=br)
    if not fused:
        mark("select")
        B.comet_scan_select(ctx, rss, k, ws.idx[:k], ws.best[:k])
    mark("classify")
    hc = ws.hit_class[: max(ev.H, 1)] if hit_class is None else hit_class
    B.comet_scan_classify(ctx, field, params, pts, nv, charge, bi, ev.wires, ev.hit_offsets,
                          ev.drift, ev.mask, hc, dca_wire=dca_wire, update_mask=update_mask,
                          n_wires=ev.W)
    mark(None)
    return ws


# kernel launches of one scan_partition call (k = 1): lattice, propagate, dca (with the selection),
# classify
LAUNCHES_PER_PARTITION = 4


class KernelTimer:
    """CUDA events between the steps of scan_partition, on the launching (current) stream."""

    def __init__(self):
        self.marks = []          # (name or None, event)

    def mark(self, name):
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        self.marks.append((name, e))

    def totals(self):
        """{step: (total ms, launches)} once the stream has been synchronised."""
        out = {}
        for (name, a), (_, b) in zip(self.marks[:-1], self.marks[1:]):
            if name is None:
                continue
            t, n = out.get(name, (0.0, 0))
            out[name] = (t + a.elapsed_time(b), n + 1)
        return out


def event_params(ev, dtype=torch.float32, stride: int = 1, lam: float = 1e-2) -> List[B.ScanParams]:
    return [params_for(sp, n, dtype, stride, lam) for sp, n in zip(ev.partitions, ev.n_steps)]


def scan_event(ctx: B.Context, field: B.DeviceField, ev, dev: DeviceEvent, ws: Workspace,
               dtype=torch.float32, stride: int = 1, lam: float = 1e-2, collect: bool = False):
    """All turn partitions of one event, in order.  With ``collect`` the per-partition best seed,
    RSS and hit classes are copied to host tensors (one synchronisation per partition)."""
    out = []
    for spec, p in zip(ev.partitions, event_params(ev, dtype, stride, lam)):
        scan_partition(ctx, field, p, spec, dev, ws)
        if collect:
            out.append(dict(idx=int(ws.idx[0]), rss=float(ws.best[0]),
                            hit_class=ws.hit_class[: dev.H].cpu().numpy().copy()))
    return out


class PipelinedScanner:
    """Scans turn partitions with the track recording of the next partition (lattice, propagate:
    they do not read the hit mask) on a second stream, beside the current partition's DCA,
    selection and classification (which read and update the mask, in partition order on the
    caller's stream; the seed of lowest RSS is selected inside the DCA launch).  Two workspaces
    alternate: a partition's recording waits only until the
    partition two back has been classified.  Every kernel is the single-event path's; the results
    are identical to scan_partition's.  With ``dca_ctas_per_sm`` the context's DCA launches leave
    room on each SM for the recording kernels to run beside them."""

    def __init__(self, ctx: B.Context, field: B.DeviceField, S: int, n_rec: int, H: int,
                 dtype=torch.float32, dca_ctas_per_sm: int = 0):
        self.ctx, self.field, self.dtype = ctx, field, dtype
        self.ws = [Workspace(S, n_rec, H, dtype) for _ in range(2)]
        self.rec = torch.cuda.Stream()
        self.free = [None, None]     # event: the workspace's last consumer (classify) finished
        self.k = 0
        ctx.set_dca_ctas_per_sm(dca_ctas_per_sm)

    def partition(self, params: B.ScanParams, spec, ev: DeviceEvent, hit_class=None,
                  rec_timer=None, timer=None, update_mask: bool = True, best_idx=None, best_rss=None):
        """Enqueues one partition (recording on the second stream, the rest on the current
        stream); returns its workspace (idx, best, rss, n_in, hit_class valid once the current
        stream reaches them).  ``best_idx`` / ``best_rss`` ([1] device tensors) take the selected
        seed and its RSS instead of the workspace's idx / best."""
        b = self.k
        self.k ^= 1
        ws = self.ws[b]
        main = torch.cuda.current_stream()
        S = spec.n_seeds
        seeds, charge, pts, nv, rss, n_in = ws.views(S, params.n_rec)
        bounds = ws.bounds[: (S + 31) // 32]
        with torch.cuda.stream(self.rec):
            if self.free[b] is not None:
                self.rec.wait_event(self.free[b])
            mark = rec_timer.mark if rec_timer is not None else (lambda name: None)
            mark("lattice")
            B.comet_scan_lattice(self.ctx, spec, seeds, charge)
            mark("propagate")
            B.comet_scan_propagate(self.ctx, self.field, params, seeds, charge, pts, nv, bounds=bounds)
            mark(None)
            ready = torch.cuda.Event()
            ready.record(self.rec)
        main.wait_event(ready)
        mark = timer.mark if timer is not None else (lambda name: None)
        mark("dca")
        bi = ws.idx[:1] if best_idx is None else best_idx
        br = ws.best[:1] if best_rss is None else best_rss
        B.comet_scan_dca(self.ctx, self.field, params, pts, nv, charge, ev.wires, ev.hit_offsets,
                         ev.drift, ev.mask, rss, n_in, n_unconverged=ws.n_unconv, n_wires=ev.W,
                         bounds=bounds, best_idx=bi, best_rss=br)
        mark("classify")
        hc = ws.hit_class[: max(ev.H, 1)] if hit_class is None else hit_class
        B.comet_scan_classify(self.ctx, self.field, params, pts, nv, charge, bi, ev.wires,
                              ev.hit_offsets, ev.drift, ev.mask, hc, update_mask=update_mask,
                              n_wires=ev.W)
        mark(None)
        done = torch.cuda.Event()
        done.record(main)
        self.free[b] = done
        return ws

    def event(self, ev, dev: DeviceEvent, params, classes=None, rec_timer=None, timer=None):
        """Every partition of an event, in order (``params`` from event_params)."""
        for p, (spec, bp) in enumerate(zip(ev.partitions, params)):
            self.partition(bp, spec, dev, hit_class=None if classes is None else classes[p],
                           rec_timer=rec_timer, timer=timer)

    def close(self):
        self.ctx.set_dca_ctas_per_sm(0)


class HostEventRunner:
    """End-to-end path from host buffers: copies an event's wires, offsets and drifts from pinned
    host memory to the device, scans every partition (one at a time, or through a PipelinedScanner),
    and copies back the per-partition best seed index, its RSS and the final hit mask.  Counts the
    bytes moved each way."""

    def __init__(self, ctx: B.Context, field: B.DeviceField, ws: Workspace, max_w: int, max_h: int,
                 dtype=torch.float32, pipeline: Optional["PipelinedScanner"] = None):
        self.ctx, self.field, self.ws, self.dtype = ctx, field, ws, dtype
        self.pipeline = pipeline
        self.dev_w = torch.zeros((6, _pad4(max_w)), dtype=dtype, device="cuda")
        self.dev_o = torch.zeros(max_w + 1, dtype=torch.int32, device="cuda")
        self.dev_d = torch.zeros(max(max_h, 1), dtype=dtype, device="cuda")
        self.dev_m = torch.zeros(max(max_h, 1), dtype=torch.uint8, device="cuda")
        self.res_idx = torch.zeros(16, dtype=torch.int64, device="cuda")
        self.res_rss = torch.zeros(16, dtype=dtype, device="cuda")
        self.h_idx = torch.zeros(16, dtype=torch.int64).pin_memory()
        self.h_rss = torch.zeros(16, dtype=dtype).pin_memory()
        self.h_mask = torch.zeros(max(max_h, 1), dtype=torch.uint8).pin_memory()

    @staticmethod
    def pin(ev, dtype=torch.float32):
        W = ev.n_wires
        w = torch.zeros((6, _pad4(W)), dtype=dtype)
        w[:, :W] = torch.as_tensor(ev.wires, dtype=dtype)
        return dict(w=w.pin_memory(), o=torch.as_tensor(ev.hit_offsets, dtype=torch.int32).pin_memory(),
                    d=torch.as_tensor(ev.drift, dtype=dtype).pin_memory(), W=W, H=ev.n_hits)

    def result_slots(self):
        """Pinned host buffers for one event's results (best seed index and RSS per partition, the
        final hit mask), so that results of events in flight are not overwritten."""
        return (torch.zeros(16, dtype=torch.int64).pin_memory(), torch.zeros(16, dtype=self.dtype).pin_memory(),
                torch.zeros(self.h_mask.numel(), dtype=torch.uint8).pin_memory())

    def run(self, ev, pinned, stride: int = 1, lam: float = 1e-2, out=None):
        """Enqueues the event on the current stream (copies in, every partition, copies out) and
        returns (bytes in, bytes out); the results land in ``out`` (``result_slots()``) or in the
        runner's own buffers once the stream reaches them."""
        W, H = pinned["W"], pinned["H"]
        ldw = pinned["w"].shape[1]
        w = self.dev_w.view(-1)[: 6 * ldw].view(6, ldw)
        w.copy_(pinned["w"], non_blocking=True)
        self.dev_o[: W + 1].copy_(pinned["o"], non_blocking=True)
        self.dev_d[:H].copy_(pinned["d"], non_blocking=True)
        self.dev_m[:H].zero_()
        dev = DeviceEvent(w, self.dev_o[: W + 1], self.dev_d[:H], self.dev_m[: max(H, 1)], W, H)
        h2d = pinned["w"].numel() * pinned["w"].element_size() + 4 * (W + 1) + \
            pinned["d"].numel() * pinned["d"].element_size()
        n = len(ev.partitions)
        for i, (spec, p) in enumerate(zip(ev.partitions, event_params(ev, self.dtype, stride, lam))):
            # the DCA launch writes the selected seed and its RSS straight into the result arrays
            bi, br = self.res_idx[i:i + 1], self.res_rss[i:i + 1]
            if self.pipeline is not None:
                self.pipeline.partition(p, spec, dev, best_idx=bi, best_rss=br)
            else:
                scan_partition(self.ctx, self.field, p, spec, dev, self.ws, best_idx=bi, best_rss=br)
        h_idx, h_rss, h_mask = out if out is not None else (self.h_idx, self.h_rss, self.h_mask)
        h_idx[:n].copy_(self.res_idx[:n], non_blocking=True)
        h_rss[:n].copy_(self.res_rss[:n], non_blocking=True)
        h_mask[:H].copy_(self.dev_m[:H], non_blocking=True)
        d2h = n * (8 + self.res_rss.element_size()) + H
        return h2d, d2h
