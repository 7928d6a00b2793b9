"""Hit-classification metrics of a scan stage (Sec. 3, "Hit classification metrics").

After a stage, the hits it classified are split by their truth turn index; the stage represents
the turn of the largest subset.  Its *efficiency* is the size of that subset over the number of
hits the represented turn induced; its *purity* is the size of that subset over the number of hits
the stage classified.  Noise hits (truth turn -1) belong to no turn: they form no subset that a
stage can represent, but they count among the classified hits (they lower the purity).  A tie
between subsets goes to the lower turn index.

These are evaluation quantities on host arrays (hit classes copied back from the device), not a
step of the scan.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class StageMetrics:
    turn: Optional[int]        # represented truth turn (None when nothing signal-like was classified)
    efficiency: float
    purity: float
    n_classified: int
    n_largest: int
    n_turn_hits: int


def stage_metrics(classified, hit_turn) -> StageMetrics:
    """Metrics of one stage from its classified-hit flags [H] and the truth turn of every hit [H]."""
    cls = np.asarray(classified).astype(bool)
    turn = np.asarray(hit_turn).astype(np.int64)
    if cls.shape != turn.shape:
        raise ValueError("classified and hit_turn must have the same shape")
    n_cls = int(cls.sum())
    sig = turn[cls]
    sig = sig[sig >= 0]
    if sig.size == 0:
        return StageMetrics(None, 0.0, 0.0, n_cls, 0, 0)
    vals, counts = np.unique(sig, return_counts=True)    # vals ascending: argmax takes the lowest
    i = int(np.argmax(counts))
    rep, largest = int(vals[i]), int(counts[i])
    n_turn = int((turn == rep).sum())
    return StageMetrics(rep, largest / n_turn, largest / n_cls, n_cls, largest, n_turn)


def event_metrics(stage_classes: Sequence, hit_turn) -> List[StageMetrics]:
    """Metrics of every stage of one event; ``stage_classes[k]`` holds the hits stage k classified."""
    return [stage_metrics(c, hit_turn) for c in stage_classes]


def average(stages: Sequence[StageMetrics]) -> dict:
    """Mean efficiency and purity over stages (a stage that classified nothing counts as 0, 0)."""
    if not stages:
        return {"efficiency": 0.0, "purity": 0.0, "n": 0}
    return {"efficiency": float(np.mean([s.efficiency for s in stages])),
            "purity": float(np.mean([s.purity for s in stages])), "n": len(stages)}
