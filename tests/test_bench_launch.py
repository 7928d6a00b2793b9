"""bench.py's multi-GPU launch on the CPU: `--gpus 2` without a launcher starts two ranks itself
(torch.distributed.run on 127.0.0.1, gloo), each takes its share of the events, and rank 0 prints
one line that reports both ranks.  `--dry-run` keeps CUDA out of it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK",
                                                            "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--dry-run", *extra],
                       capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_bench_spawns_two_ranks_and_reports_both():
    out = _run("--gpus", "2", "--steps", "3", "--warmup", "1")
    assert out["n_gpus"] == 2 and out["dry_run"]
    ranks = sorted(out["ranks"], key=lambda r: r["rank"])
    assert [r["rank"] for r in ranks] == [0, 1]
    assert [r["local_rank"] for r in ranks] == [0, 1]
    ev0, ev1 = set(ranks[0]["events"]), set(ranks[1]["events"])
    assert len(ev0) == len(ev1) == 3 and not ev0 & ev1      # disjoint events, weak scaling
    assert out["events_timed"] == 6


def test_bench_single_rank_dry_run():
    out = _run("--steps", "2", "--warmup", "1")
    assert out["n_gpus"] == 1 and len(out["ranks"]) == 1 and out["events_timed"] == 2
