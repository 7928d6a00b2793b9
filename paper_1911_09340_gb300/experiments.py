"""Studies built on the scan (the evaluation side of the paper's Sec. 3, on synthetic events).

    python -m paper_1911_09340_gb300.experiments lambda-sweep [--events N] [--stride s]
    python -m paper_1911_09340_gb300.experiments backward [--events N] [--stride s]

* ``lambda-sweep``: hit-classification efficiency and purity (metrics.py) of the first stage and of
  all stages as the cutoff lambda runs over 0.5-1.2 mm in 0.1 mm steps (the range of the paper's
  cutoff optimisation, Sec. 3.2; there the first stage is the last turn, here it is the first turn
  from the vertex, and there is no DAF fit or self-refining after the scan).
* ``backward``: the first stage scanned forwards from the start of the turn and backwards from its
  end with the charge and momentum flipped (the paper's two half tracks, Sec. 3.1), each over the
  whole turn.

Every scan runs through the library's kernels (scan.scan_partition); only the metrics are computed
on the host from the copied-back hit classes.  One JSON line per result.
"""
from __future__ import annotations

import argparse
import json
import sys
from typing import List, Sequence

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


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["lambda-sweep", "backward"])
    ap.add_argument("--events", type=int, default=32)
    ap.add_argument("--stride", type=int, default=16)
    ap.add_argument("--lambda-mm", type=float, default=10.0, help="cutoff of the backward study")
    args = ap.parse_args(argv)
    if args.study == "lambda-sweep":
        rows = lambda_sweep(args.events, stride=args.stride)
    else:
        rows = backward_study(args.events, args.stride, args.lambda_mm * 1e-3)
    for r in rows:
        print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
