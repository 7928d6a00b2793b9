"""Host-side sharding for several GPUs (one process per GPU).

Events are independent, so the natural split is by event: rank r takes events r, r + N, r + 2N, ...
and no data crosses ranks.  A single turn partition can also be split by seed range; the only
exchange is then the merge of each shard's k best (RSS, seed index) pairs, under the same order as
comet_scan_select (ascending RSS, ties by lowest seed index, NaN last).
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple


def event_indices(n: int, rank: int, world: int, start: int = 0) -> List[int]:
    """The n events of rank `rank` out of `world`: start + rank, start + rank + world, ..."""
    return [start + rank + world * i for i in range(n)]


def shard_range(total: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [begin, end) share of `total` items for `rank`; shares differ by at most one."""
    base, extra = divmod(total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def _key(v: float, i: int):
    nan = isinstance(v, float) and math.isnan(v)
    return (nan, 0.0 if nan else v, i)


def merge_topk(values: Sequence[Sequence[float]], indices: Sequence[Sequence[int]], k: int):
    """Merge per-shard candidate lists (global seed indices) into the global k best."""
    pairs = [(float(v), int(i)) for vs, ix in zip(values, indices) for v, i in zip(vs, ix)]
    pairs.sort(key=lambda p: _key(*p))
    best = pairs[:k]
    return [i for _, i in best], [v for v, _ in best]


def allgather_topk(local_values, local_indices, k: int, group=None):
    """Gather every rank's candidates (torch.distributed, any backend) and merge them."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    buf = [None] * world
    dist.all_gather_object(buf, (list(map(float, local_values)), list(map(int, local_indices))),
                           group=group)
    return merge_topk([b[0] for b in buf], [b[1] for b in buf], k)
