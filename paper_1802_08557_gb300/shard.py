"""Multi-GPU sharding of one LP batch: the LPs are independent (Section 4.1
assigns each LP its own block and no data moves between LPs), so N ranks
split the batch into contiguous LP ranges and solve them with no exchange on
the data path.  The only cross-rank step is gathering the per-rank results.

Ranges are balanced by the estimated work of each LP, (m+1)(n+1)(m+n): a
pivot updates the (m+1)(n+1) condensed tableau and the simplex method takes
O(m+n) pivots on random dense LPs.
"""
from __future__ import annotations

import numpy as np


def work_estimate(m, n) -> np.ndarray:
    m = np.asarray(m, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    return (m + 1.0) * (n + 1.0) * (m + n)


def shard_bounds(m, n, world_size: int) -> np.ndarray:
    """Boundaries b[0] = 0 <= b[1] <= ... <= b[world_size] = num_lps; rank r
    solves LPs b[r] .. b[r+1]-1.  Rank r's range ends at the first LP whose
    work prefix reaches (r+1)/world_size of the total, so every range holds
    about the same work; the split depends only on the sizes."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    w = work_estimate(m, n)
    num = w.size
    bounds = np.zeros(world_size + 1, dtype=np.int64)
    bounds[-1] = num
    if num == 0:
        return bounds
    prefix = np.cumsum(w)
    total = prefix[-1]
    for r in range(1, world_size):
        # first index whose inclusive prefix reaches the target, +1
        cut = int(np.searchsorted(prefix, total * r / world_size, side="left")) + 1
        bounds[r] = min(max(cut, bounds[r - 1]), num)
    return bounds


def local_range(m, n, rank: int, world_size: int) -> tuple[int, int]:
    b = shard_bounds(m, n, world_size)
    return int(b[rank]), int(b[rank + 1])


def solve_sharded(batch, solve_fn, rank: int, world_size: int, group=None) -> dict:
    """Solve this rank's range of ``batch`` with ``solve_fn`` (a callable that
    takes an LPBatch and returns dict(status, iters, obj, x, y) in the batch
    layout) and gather every rank's results, in LP order, on every rank.

    ``group`` is a torch.distributed process group (None: the default group);
    with world_size == 1 nothing is exchanged."""
    lo, hi = local_range(batch.m, batch.n, rank, world_size)
    part = solve_fn(batch.subset(np.arange(lo, hi))) if hi > lo else None
    local = {"rank": rank, "lo": lo, "hi": hi}
    if part is not None:
        for key in ("status", "iters", "obj", "x", "y"):
            local[key] = np.asarray(part[key])
    if world_size == 1:
        parts = [local]
    else:
        import torch.distributed as dist
        parts = [None] * world_size
        dist.all_gather_object(parts, local, group=group)
    parts.sort(key=lambda p: p["lo"])
    out = {"status": [], "iters": [], "obj": [], "x": [], "y": []}
    expect = 0
    for p in parts:
        if p["lo"] != expect:
            raise RuntimeError(f"shard ranges do not tile the batch: rank {p['rank']} starts at {p['lo']}")
        expect = p["hi"]
        if p["hi"] > p["lo"]:
            for key in out:
                out[key].append(p[key])
    if expect != batch.num_lps:
        raise RuntimeError(f"shard ranges end at {expect}, batch has {batch.num_lps} LPs")
    return {key: (np.concatenate(v) if v else np.zeros(0)) for key, v in out.items()}
