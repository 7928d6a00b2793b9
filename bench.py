"""Benchmark of the seed scan on synthetic multi-turn drift-chamber events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--stride s]

A step is one event of the 1000-event FP32 workload (2-5 turns, p ~ U(100, 105) MeV/c, 17 vertex
disks, 60-250 fired wires plus 10% noise hits, 2^18 seeds per turn partition, uniform 1 T field):
every turn partition runs lattice -> propagate -> dca -> select -> classify -> mask update.  The
metric is seed x hit DCA evaluations per second: for each partition, seeds times hits still unmasked
when the partition is scanned.  Events are independent, so N GPUs take disjoint events (weak
scaling, no data-path collective).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "seed x hit DCA evals/s"
WORKLOAD = ("multi-turn electron events (2-5 turns, 100-105 MeV/c), 2^18 seeds per turn partition "
            "(16x16x32x32), uniform 1 T, 18-layer stereo chamber")
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""
        else:
            self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def make_events(indices, counts=(16, 16, 32, 32)):
    from paper_1911_09340_gb300 import synth
    ch = synth.make_chamber()
    return [synth.multi_turn_event(i, ch, counts=tuple(counts)) for i in indices]


def evals_of(ev, classes):
    """Seed x unmasked-hit pairs of each partition, from the per-partition hit classes."""
    return pairs_of(ev, classes)[0]


def pairs_of(ev, classes):
    """(seed x unmasked hit, seed x wire with an unmasked hit) pairs summed over the partitions."""
    H = ev.n_hits
    masked = np.zeros(H, bool)
    hits = wires = 0
    offs = np.asarray(ev.hit_offsets)
    for spec, cls in zip(ev.partitions, classes):
        live = ~masked
        hits += spec.n_seeds * int(live.sum())
        csum = np.concatenate([[0], np.cumsum(live.astype(np.int64))])
        per_wire = csum[offs[1:]] - csum[offs[:-1]]          # unmasked hits of each wire
        wires += spec.n_seeds * int((per_wire > 0).sum())
        masked |= cls[:H].astype(bool)
    return hits, wires


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline of our arm, and the whole reference arm)
# ------------------------------------------------------------------------------------------------

def oracle_rate(ev, target_s: float = 10.0, nthreads=None, stride: int = 16):
    """Times the oracle's RSS scan of partition 0 on a strided sample of its seeds, sized for
    ~target_s of CPU time, recording every stride-th state like the GPU arm; returns (evals/s,
    threads, sample description, wall seconds of the timed sample)."""
    import oracle as O
    from paper_1911_09340_gb300 import synth
    nthreads = nthreads or O.default_threads()
    spec = ev.partitions[0]
    seeds = O.lattice(spec).astype(np.float32).astype(np.float64)
    op = O.Params(n_steps=ev.n_steps[0], stride=stride, lam=0.01, tol=1e-12)
    field = synth.uniform_field(1.0)
    wires = O.wires_aos(ev.wires)
    mask = np.zeros(ev.n_hits, np.uint8)

    def run(n):
        sub = seeds[:: max(1, spec.n_seeds // n)][:n]
        t0 = time.perf_counter()
        O.scan(field, op, sub, spec.charge, wires, ev.hit_offsets, ev.drift, mask, nthreads=nthreads)
        return time.perf_counter() - t0, sub.shape[0]

    dt, n = run(max(nthreads * 8, 64))
    n2 = int(min(spec.n_seeds, max(n, n * target_s / max(dt, 1e-3))))
    dt, n = run(n2)
    evals = n * ev.n_hits
    return evals / dt, nthreads, f"{n} of {spec.n_seeds} seeds (strided) of turn partition 0 of event 0, " \
                                f"{ev.n_hits} hits, stride {stride}, FP64 oracle, {dt:.1f} s", dt


def workload_config(args, arithmetic: str):
    """The workload keys both arms report; ``arithmetic`` names the precision the arm computes in
    (the events, lattice and parameters are the same)."""
    counts = args.lattice or (16, 16, 32, 32)
    return {"workload": WORKLOAD, "arithmetic": arithmetic,
            "seeds_per_partition": int(np.prod(counts)), "stride": args.stride,
            "lambda_m": 0.01, "rk4_step_m": 1e-3}


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    ev = make_events([0])[0]
    steps, walls = [], []
    for i in range(args.warmup + args.steps):
        rate, cores, sample, wall = oracle_rate(ev, target_s=args.ref_seconds, stride=args.stride)
        if i >= args.warmup:
            steps.append(rate)
            walls.append(wall)
    value = statistics.median(steps)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "ms_per_step": 1e3 * statistics.mean(walls),   # a step: one bounded sample (see cpu_baseline)
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args, "FP64 CPU oracle"), parallelism=f"host threads ({cores})"),
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------------------------------------
# Our arm
# ------------------------------------------------------------------------------------------------

def run_ours(args, rank, world):
    import torch

    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import scan, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ctx = B.Context(local)
    if args.only_legs:
        # profiling: the two extra configurations alone
        if rank == 0:
            print(json.dumps({"legs": {
                "single_event_fp64": leg_single_event_fp64(ctx, reps=args.fp64_reps),
                "table_field_fp32": leg_table_field_fp32(ctx, 2, args.table_events, args.stride)},
                "note": "profiling run (--only-legs)"}), flush=True)
        ctx.close()
        return
    field = B.DeviceField.from_synth(synth.uniform_field(1.0))
    dtype = torch.float32
    n_ev = args.warmup + args.steps
    from paper_1911_09340_gb300 import multi
    idx = multi.event_indices(n_ev, rank, world)
    events = make_events(idx, args.lattice)
    max_rec = max(n // args.stride + 1 for ev in events for n in ev.n_steps)
    max_h = max(ev.n_hits for ev in events)
    max_w = max(ev.n_wires for ev in events)
    S = events[0].partitions[0].n_seeds
    pipelined = not args.sequential
    if pipelined:
        # the next partition's lattice + propagate on a second stream beside the current
        # partition's dca / select / classify (two workspaces; identical results)
        pipe = scan.PipelinedScanner(ctx, field, S, max_rec, max_h, dtype)
        ws = pipe.ws[0]
    else:
        pipe = None
        ws = scan.Workspace(S, max_rec, max_h, dtype)
    devs = [scan.DeviceEvent.from_event(ev, dtype) for ev in events]
    classes = [torch.zeros((len(ev.partitions), max(ev.n_hits, 1)), dtype=torch.uint8, device="cuda")
               for ev in events]
    params = [scan.event_params(ev, dtype, stride=args.stride) for ev in events]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    timer = scan.KernelTimer()
    rec_timer = scan.KernelTimer()

    def step(i, t=None, rt=None):
        ev, dev = events[i], devs[i]
        if pipe is not None:
            pipe.event(ev, dev, params[i], classes=classes[i], rec_timer=rt, timer=t)
            return
        for p, (spec, bp) in enumerate(zip(ev.partitions, params[i])):
            scan.scan_partition(ctx, field, bp, spec, dev, ws, hit_class=classes[i][p], timer=t)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    gpu = torch.cuda.current_device()
    with ClockSampler(gpu) as clk:
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        if pipe is not None:
            # back to back: the timed region is one interval on the stream; the recording stream
            # starts inside it (the track points, 0.44 GB per partition, exceed L2)
            t0.record()
            pipe.rec.wait_event(t0)
            for j in range(args.steps):
                step(args.warmup + j, timer, rec_timer)
                ends[j].record()
        else:
            for j in range(args.steps):
                flush.fill_(j & 0xFF)                     # evict L2 between steps (not timed)
                starts[j].record()
                step(args.warmup + j, timer)
                ends[j].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier(world)
    if pipe is not None:
        # per event: completion to completion (the events overlap on the recording stream)
        marks = [t0] + ends
        step_ms = [a.elapsed_time(b) for a, b in zip(marks[:-1], marks[1:])]
    else:
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_s = sum(step_ms) / 1e3
    evals = 0
    wire_pairs = 0
    n_parts = 0
    for j in range(args.steps):
        i = args.warmup + j
        ev = events[i]
        cl = classes[i].cpu().numpy()
        e_h, e_w = pairs_of(ev, cl)
        evals += e_h
        wire_pairs += e_w
        n_parts += len(ev.partitions)
    kt = dict(timer.totals())
    kt.update(rec_timer.totals())
    t_max = max_over_ranks(dev_s, world)
    evals_all = sum_over_ranks(float(evals), world)
    events_all = args.steps * world
    value = evals_all / t_max
    clocks = clk.summary()

    # ---- end to end through host buffers (pinned), copies inside the timed region
    if args.no_e2e:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "evals/s",
                              "kernel_ms": {k: round(v[0], 3) for k, v in kt.items()},
                              "clocks": clocks, "note": "profiling run (--no-e2e)"}), flush=True)
        return
    # Like the device leg, the host enqueues event after event and synchronises once at the end;
    # each event's timed region holds its host->device copies, its partitions and the
    # device->host copy of its results into its own pinned slots.
    runner = scan.HostEventRunner(ctx, field, ws, max_w, max_h, dtype, pipeline=pipe)
    pinned = [runner.pin(ev, dtype) for ev in events]
    slots = [runner.result_slots() for _ in range(args.steps)]
    for i in range(args.warmup):
        runner.run(events[i], pinned[i], stride=args.stride)
    torch.cuda.synchronize()
    barrier(world)
    e_starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    h2d = d2h = 0
    e0 = torch.cuda.Event(enable_timing=True)
    if pipe is not None:
        e0.record()
        pipe.rec.wait_event(e0)
    for j in range(args.steps):
        i = args.warmup + j
        if pipe is None:
            flush.fill_(j & 0xFF)                     # evict L2 between events (not timed)
            e_starts[j].record()
        b_in, b_out = runner.run(events[i], pinned[i], stride=args.stride, out=slots[j])
        e_ends[j].record()
        h2d += b_in
        d2h += b_out
    torch.cuda.synchronize()
    if pipe is not None:
        e2e_ms = e0.elapsed_time(e_ends[-1])
    else:
        e2e_ms = sum(a.elapsed_time(b) for a, b in zip(e_starts, e_ends))
    for j in range(args.steps):
        # the results read back are the device leg's: the final mask holds every classified hit
        i = args.warmup + j
        H = events[i].n_hits
        want = classes[i][:, :H].any(0).cpu().numpy()
        if not np.array_equal(slots[j][2][:H].numpy().astype(bool), want):
            raise RuntimeError(f"end-to-end results of event {i} differ from the device leg's")
    barrier(world)
    e2e_t = max_over_ranks(e2e_ms / 1e3, world)
    e2e_value = evals_all / e2e_t

    if rank != 0:
        return
    # ---- roofline of the dominant kernel
    peaks = _peaks()
    dca_flops = (DCA_FLOPS_PER_WIRE * wire_pairs + DCA_FLOPS_PER_HIT * evals) / max(n_parts, 1)
    # states the timed propagate launches recorded (tracks leaving the target region stop early):
    # lattice + propagate of each timed partition once more, untimed, summing n_valid
    recorded = 0
    for j in range(args.steps):
        i = args.warmup + j
        for spec, bp in zip(events[i].partitions, params[i]):
            seeds, charge, pts, nv, _, _ = ws.views(spec.n_seeds, bp.n_rec)
            B.comet_scan_lattice(ctx, spec, seeds, charge)
            B.comet_scan_propagate(ctx, field, bp, seeds, charge, pts, nv)
            recorded += int(nv.sum().item())
    prop_bytes = (PROP_BYTES_PER_REC * recorded + 24 * S * n_parts) / max(n_parts, 1)
    survey = survey_count_entry(kt["dca"][0] / kt["dca"][1], evals / max(n_parts, 1), clocks, peaks)
    # the same kernels once more, one partition at a time on one stream (not part of `value`): the
    # DCA kernel's duration without the recording kernels of the next partition beside it
    seq_roof = None
    if pipe is not None:
        seq_timer = scan.KernelTimer()
        for j in range(args.steps):
            i = args.warmup + j
            devs[i].mask.zero_()
            for p, (spec, bp) in enumerate(zip(events[i].partitions, params[i])):
                flush.fill_((i + p) & 0xFF)
                scan.scan_partition(ctx, field, bp, spec, devs[i], ws, timer=seq_timer)
        torch.cuda.synchronize()
        skt = seq_timer.totals()
        seq_roof = {"dca": roofline_entry("dca", skt["dca"][0] / skt["dca"][1], prop_bytes, clocks, peaks,
                                          dca_flops, args.stride),
                    "dca_survey_count": survey_count_entry(skt["dca"][0] / skt["dca"][1],
                                                           evals / max(n_parts, 1), clocks, peaks),
                    "propagate": roofline_entry("propagate", skt["propagate"][0] / skt["propagate"][1],
                                                prop_bytes, clocks, peaks, dca_flops, args.stride),
                    "kernel_ms": {k: round(v[0], 3) for k, v in skt.items()},
                    "note": "the timed events once more, one partition at a time on one stream, "
                            "a 256 MiB buffer written before each partition; not part of value"}
    # the dominant kernel by device time, one partition at a time (in the pipelined region the
    # recording's interval on its stream spans the DCA launch it runs beside)
    share = skt if pipe is not None else kt
    dom = max(share, key=lambda k: share[k][0])
    roof = roofline_entry(dom, kt[dom][0] / kt[dom][1], prop_bytes, clocks, peaks, dca_flops,
                          args.stride)
    second = "propagate" if dom != "propagate" else "dca"
    roof_prop = roofline_entry(second, kt[second][0] / kt[second][1], prop_bytes, clocks, peaks,
                               dca_flops, args.stride)
    cpu = (oracle_rate(make_events([0])[0], target_s=args.cpu_seconds, stride=args.stride)
           if not args.no_cpu else None)
    cpu1 = (oracle_rate(make_events([0])[0], target_s=max(1.0, args.cpu_seconds / 4), nthreads=1,
                        stride=args.stride) if not args.no_cpu else None)
    out = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "events_per_s": events_all / t_max,
        "event_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                     "max": max(step_ms)},
        "config": dict(workload_config(args, "FP32 GPU"), events=events_all, partitions=n_parts * world,
                       l2=("inputs larger than L2: the track points of each partition (0.44 GB; "
                           "two workspaces alternate) are written and read inside every step"
                           if pipe is not None else
                           "256 MiB buffer written between timed steps; track points (~0.44 GB "
                           "per partition) also exceed L2"),
                       schedule=("pipelined: lattice + propagate of partition p+1 on a second stream "
                                 "beside partition p's dca / select / classify"
                                 if pipe is not None else "sequential: one partition at a time"),
                       parallelism=f"replicas: {world} GPU(s), disjoint events"),
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": scan.LAUNCHES_PER_PARTITION * n_parts,
        "kernel_ms": {k: round(v[0], 3) for k, v in kt.items()},
        "roofline": roof,
        "roofline_survey_count": survey,
        "roofline_sequential": seq_roof,
        "roofline_other": roof_prop,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
        "wall_s": wall,
    }
    if cpu is not None:
        out["cpu_baseline"] = {"value": cpu[0], "unit": "evals/s", "cores": cpu[1], "kind": "oracle",
                               "sample": cpu[2], "value_1_thread": cpu1[0],
                               "sample_1_thread": cpu1[2]}
    if not args.no_legs:
        del ws, devs, runner
        if pipe is not None:
            pipe.close()
            del pipe
        torch.cuda.empty_cache()
        out["legs"] = {
            "single_event_fp64": leg_single_event_fp64(ctx, reps=args.fp64_reps),
            "table_field_fp32": leg_table_field_fp32(ctx, 2, args.table_events, args.stride),
        }
    print(json.dumps(out), flush=True)
    ctx.close()


# ------------------------------------------------------------------------------------------------
# Extra legs: the paper's precision on the single-event configuration, and the tabulated field
# ------------------------------------------------------------------------------------------------

def _time_events(run_event, n_warm: int, n_timed: int):
    """Runs n_warm untimed then n_timed timed events (CUDA events around each on the current
    stream); returns per-event ms and the KernelTimer totals of one more pass over the timed ones."""
    import torch

    from paper_1911_09340_gb300 import scan
    for i in range(n_warm):
        run_event(i, None)
    torch.cuda.synchronize()
    st = [torch.cuda.Event(enable_timing=True) for _ in range(n_timed)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(n_timed)]
    for j in range(n_timed):
        st[j].record()
        run_event(n_warm + j, None)
        en[j].record()
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in zip(st, en)]
    timer = scan.KernelTimer()
    for j in range(n_timed):
        run_event(n_warm + j, timer)
    torch.cuda.synchronize()
    return ms, timer.totals()


def leg_single_event_fp64(ctx, reps: int, stride: int = 1):
    """The paper's precision (FP64, Sec. 2.2) on the single-event configuration: one 104 MeV/c
    electron at 80 degrees to the axis making 2 turns in a uniform 1 T field, 8^4 seeds per turn
    partition, RK4 step 1 mm, every state recorded (Algorithm 1), lambda = 1 cm.  The event is
    repeated `reps` times (the mask reset before each); per-event CUDA-event times."""
    import torch

    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import scan, synth
    dt = torch.float64
    ev = synth.single_event_fp64()
    field = B.DeviceField.from_synth(synth.uniform_field(1.0))
    dev = scan.DeviceEvent.from_event(ev, dt)
    params = scan.event_params(ev, dt, stride=stride)
    ws = scan.Workspace(ev.partitions[0].n_seeds, max(p.n_rec for p in params), ev.n_hits, dt)
    classes = torch.zeros((len(ev.partitions), max(ev.n_hits, 1)), dtype=torch.uint8, device="cuda")

    def run_event(_i, t):
        dev.mask.zero_()
        for p, (spec, bp) in enumerate(zip(ev.partitions, params)):
            scan.scan_partition(ctx, field, bp, spec, dev, ws, hit_class=classes[p], timer=t)

    ms, kt = _time_events(run_event, 3, reps)
    hits, wires = pairs_of(ev, classes.cpu().numpy())
    mean_ms = sum(ms) / len(ms)
    n_parts = len(ev.partitions)
    dca_ms = kt["dca"][0] / kt["dca"][1]
    flops = (DCA_FLOPS_PER_WIRE * wires + DCA_FLOPS_PER_HIT * hits) / n_parts
    tf = flops / (dca_ms * 1e-3) / 1e12
    return {
        "config": "one 104 MeV/c electron at 80 deg, 2 turns, uniform 1 T; 8^4 seeds per turn "
                  f"partition; RK4 step 1 mm, stride {stride}; lambda 1 cm; {ev.n_hits} hits on "
                  f"{ev.n_wires} wires",
        "dtype": "f64", "events": reps, "evals_per_s": hits / (mean_ms * 1e-3),
        "events_per_s": 1e3 / mean_ms,
        "event_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "kernel_ms_per_event": {k: round(v[0] / reps, 4) for k, v in kt.items()},
        "gpu_launches_per_event": scan.LAUNCHES_PER_PARTITION * n_parts,
        "roofline": {"kernel": "dca", "bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS, "traffic": None,
                     "peak_source": "nominal FP64 rate of the part (not measured)",
                     "flops_per_launch": flops, "avg_launch_ms": dca_ms},
    }


def leg_table_field_fp32(ctx, n_warm: int, n_timed: int, stride: int):
    """The non-uniform field (FP32): events with the DIO-shaped momentum spectrum (50-105 MeV/c),
    the harmonic solenoid model (1 T centre, 5% gradients) tabulated on a 5 mm grid and
    interpolated trilinearly at every RK4 stage, 2^18 seeds per turn partition."""
    import torch

    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import scan, synth
    dt = torch.float32
    fld = synth.table_field()
    events = [synth.table_field_event(i, fld) for i in range(n_warm + n_timed)]
    field = B.DeviceField.from_synth(fld, interleaved=True)
    S = max(sp.n_seeds for ev in events for sp in ev.partitions)
    params = [scan.event_params(ev, dt, stride=stride) for ev in events]
    ws = scan.Workspace(S, max(p.n_rec for ps in params for p in ps), max(ev.n_hits for ev in events), dt)
    devs = [scan.DeviceEvent.from_event(ev, dt) for ev in events]
    classes = [torch.zeros((len(ev.partitions), max(ev.n_hits, 1)), dtype=torch.uint8, device="cuda")
               for ev in events]

    def run_event(i, t):
        devs[i].mask.zero_()
        for p, (spec, bp) in enumerate(zip(events[i].partitions, params[i])):
            scan.scan_partition(ctx, field, bp, spec, devs[i], ws, hit_class=classes[i][p], timer=t)

    ms, kt = _time_events(run_event, n_warm, n_timed)
    hits = n_parts = 0
    steps = 0
    for i in range(n_warm, n_warm + n_timed):
        hits += pairs_of(events[i], classes[i].cpu().numpy())[0]
        n_parts += len(events[i].partitions)
        # RK4 steps the recording took: (states recorded - 1) x stride per seed
        for spec, bp in zip(events[i].partitions, params[i]):
            seeds, charge, pts, nv, _, _ = ws.views(spec.n_seeds, bp.n_rec)
            B.comet_scan_lattice(ctx, spec, seeds, charge)
            B.comet_scan_propagate(ctx, field, bp, seeds, charge, pts, nv)
            steps += int((nv.long() - 1).sum().item()) * bp.stride
    tot_ms = sum(ms)
    prop_ms = kt["propagate"][0] / kt["propagate"][1]
    flops = TABLE_FLOPS_PER_STEP * steps / n_parts
    tf = flops / (prop_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops(_peaks())
    return {
        "config": "DIO-shaped momenta 50-105 MeV/c, tabulated solenoid field (5 mm grid, trilinear, "
                  f"[nz][ny][nx][4] float32), 2^18 seeds per turn partition, stride {stride}, "
                  "lambda 1 cm",
        "dtype": "f32", "events": n_timed, "partitions": n_parts,
        "momenta_MeV": [round(float(np.hypot(events[i].pt, events[i].pz)), 1)
                        for i in range(n_warm, n_warm + n_timed)],
        "evals_per_s": hits / (tot_ms * 1e-3), "events_per_s": n_timed / (tot_ms * 1e-3),
        "event_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "kernel_ms": {k: round(v[0], 3) for k, v in kt.items()},
        "gpu_launches": scan.LAUNCHES_PER_PARTITION * n_parts,
        "roofline": {"kernel": "propagate", "bound": "alu", "achieved": tf, "peak": peak,
                     "unit": "TFLOP/s", "frac": tf / peak, "traffic": None,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
                     "flops_per_launch": flops, "flops_per_rk4_step": TABLE_FLOPS_PER_STEP,
                     "avg_launch_ms": prop_ms},
    }


# Algorithmic work of the kernels (counted from the formulas; FMA = 2 flops):
#  - per (seed, wire with an unmasked hit), Algorithm 2 from the closest recorded state: 3
#    virtual-plane evaluations (35 flops each), 2 RK4 refinement steps in the axial-field map (38
#    each) and the DCA (20) = 201 FP32 flops; per (seed, unmasked hit) the residual, min, cap,
#    square and accumulate of Eq. 1 = 8 flops.  The closest-state search is not counted;
#  - the recording of one state: 6 FP32 stores = 24 bytes (the propagate kernel is store-bound),
#    counted over the states actually recorded (sum of n_valid), plus 24 bytes per seed read.
#  - one RK4 step in a tabulated field: 4 trilinear lookups x (cell coordinates and weights 9 +
#    3 components x 7 linear interpolations x 3 flops = 72) + 4 derivative evaluations x 15
#    (dx/ds 3, p x B 9, scale 3) + 3 intermediate states x 6 FMA (36) + the combination
#    k1 + 2 k2 + 2 k3 + k4 of 6 components (54) = 438 FP32 flops;
#  - FP64 peak: the part's nominal FP64 rate (1.25 TFLOP/s), not measured.
DCA_FLOPS_PER_WIRE = 201
DCA_FLOPS_PER_HIT = 8
PROP_BYTES_PER_REC = 24
TABLE_FLOPS_PER_STEP = 438
INSTR_PER_EVAL_ESTIMATE = 285
FP64_PEAK_TFLOPS = 1.25

# DRAM bytes (read + write) per launch of the two main kernels on this workload at stride 32, from a
# one-pass ncu launch list of `python bench.py --no-cpu --no-legs` (dram__bytes_read.sum +
# dram__bytes_write.sum, mean over its 108 DCA launches and 136 propagate launches: warm-up, timed,
# end-to-end and one-at-a-time passes, plus one untimed lattice + propagate per timed partition to
# count the recorded states).
# Valid only for the kernel sources they were measured on (SHA-1 of the package's csrc/ files);
# reported as null once those change.
NCU_TRAFFIC = {"csrc_sha1": "4e3dd4393e52b4d843f8a1d7b3ca6aaa9c6a8301", "stride": 32,
               "dca": 171.5e6, "propagate": 403.7e6}


def csrc_sha1() -> str:
    import hashlib
    d = os.path.join(ROOT, "paper_1911_09340_gb300", "csrc")
    h = hashlib.sha1()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel: str, stride: int):
    try:
        ok = csrc_sha1() == NCU_TRAFFIC["csrc_sha1"] and stride == NCU_TRAFFIC["stride"]
    except OSError:
        ok = False
    return NCU_TRAFFIC.get(kernel) if ok else None


def survey_count_entry(avg_ms, evals_per_launch, clocks, peaks):
    """The DCA kernel against the FP32 instruction peak by an a-priori instruction count: 285 FP32
    instructions (the middle of a 250-320 estimate: 2-3 Newton iterations of an RK4 partial step and
    the plane and distance arithmetic, plus min / cap / square) per DCA evaluation, i.e. per (seed,
    unmasked hit) pair, against 152 SMs x 128 FP32 lanes x the maximum SM clock."""
    instr = INSTR_PER_EVAL_ESTIMATE * evals_per_launch
    rate = instr / (avg_ms * 1e-3)
    peak = 152 * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    return {"kernel": "dca", "bound": "alu", "achieved": rate / 1e12, "peak": peak / 1e12,
            "unit": "T FP32 instr/s", "frac": rate / peak, "instr_per_eval": INSTR_PER_EVAL_ESTIMATE,
            "evals_per_launch": evals_per_launch, "avg_launch_ms": avg_ms,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x max SM clock"}


def fp32_peak_tflops(peaks):
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x the maximum SM clock."""
    return 2 * 152 * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def roofline_entry(kernel, avg_ms, prop_bytes_per_launch, clocks, peaks, dca_flops_per_launch,
                   stride=None):
    traffic = measured_traffic(kernel, stride)
    if kernel == "propagate":
        bytes_ = prop_bytes_per_launch
        gbs = bytes_ / (avg_ms * 1e-3) / 1e9
        hbm = peaks.get("hbm_gbs", 6782.8)
        return {"kernel": kernel, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "traffic": traffic, "algorithmic_bytes": bytes_,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    if kernel == "dca":
        tf = dca_flops_per_launch / (avg_ms * 1e-3) / 1e12
        peak = fp32_peak_tflops(peaks)
        return {"kernel": kernel, "bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                "frac": tf / peak, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
                "flops_per_launch": dca_flops_per_launch,
                "flops_per_unit": {"seed_wire": DCA_FLOPS_PER_WIRE, "seed_hit": DCA_FLOPS_PER_HIT},
                "avg_launch_ms": avg_ms}
    return {"kernel": kernel, "bound": None, "achieved": None, "peak": None, "unit": None,
            "frac": None, "traffic": None, "avg_launch_ms": avg_ms}


def run_dry(args, rank, world):
    """--dry-run: the launch, sharding and reduction logic without CUDA (gloo ranks on the CPU):
    each rank takes its events as in a real run, and rank 0 prints one line with what every rank
    reported."""
    from paper_1911_09340_gb300 import multi
    idx = multi.event_indices(args.warmup + args.steps, rank, world)
    mine = {"rank": rank, "events": idx[args.warmup:], "local_rank": int(os.environ.get("LOCAL_RANK", "0"))}
    if world > 1:
        import torch.distributed as dist
        got = [None] * world
        dist.all_gather_object(got, mine)
    else:
        got = [mine]
    total = sum_over_ranks(float(len(mine["events"])), world)
    if rank == 0:
        print(json.dumps({"metric": METRIC, "dry_run": True, "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "events_timed": total, "ranks": got}), flush=True)


def spawn_ranks(n: int) -> int:
    """`--gpus N` without a launcher: start N ranks of this script (one per GPU) under
    torch.distributed.run on this node and return its exit status; rank 0 prints the line."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--stride", type=int, default=32,
                    help="record every stride-th RK4 state (h = 1 mm is unchanged)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling)")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the single-event FP64 and table-field legs")
    ap.add_argument("--fp64-reps", type=int, default=20, help="timed events of the FP64 leg")
    ap.add_argument("--only-legs", action="store_true",
                    help="run only the FP64 single-event and table-field legs (profiling)")
    ap.add_argument("--table-events", type=int, default=3, help="timed events of the table-field leg")
    ap.add_argument("--sequential", action="store_true",
                    help="one partition at a time on one stream (no recording beside the DCA)")
    ap.add_argument("--dry-run", action="store_true",
                    help="no CUDA: exercise the rank launch, sharding and reductions on the CPU")
    ap.add_argument("--lattice", type=lambda s: [int(x) for x in s.split(",")],
                    default=[16, 16, 32, 32], help="seed lattice counts (z0,phi,pz,pt); "
                    "the workload is 16,16,32,32, smaller lattices are for profiling only")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args.gpus))
    rank, world = dist_setup(args.gpus)
    if args.dry_run:
        run_dry(args, rank, world)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
