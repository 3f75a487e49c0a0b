"""Event sharding over ranks (one process per GPU).

Events are independent, so the finding work splits by whole events with no
exchange on the data path: rank r of a world of size W processes its own events,
and only timing figures are combined (max of the per-rank step times, sum of the
units), through torch.distributed collectives on small tensors.
"""
from __future__ import annotations

import torch


def events_for_rank(rank: int, world: int, per_rank: int, first: int = 0) -> list[int]:
    """Weak scaling: every rank gets its own block of `per_rank` event ids."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("bad rank/world/per_rank")
    start = first + rank * per_rank
    return list(range(start, start + per_rank))


def split_events(n_events: int, rank: int, world: int) -> range:
    """Strong scaling: a fixed set of events divided into contiguous, near-equal shards."""
    if not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_events, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def event_costs(event_offsets, seed_event, bins_per_event: int):
    """Estimated finding cost of each event: its seeds times (1 + the mean number
    of hits per bin), i.e. seeds times the hits a window of a few bins holds."""
    import numpy as np
    evo = np.asarray(event_offsets, dtype=np.int64)
    n_ev = evo.shape[0] - 1
    seeds = np.bincount(np.asarray(seed_event, dtype=np.int64), minlength=n_ev)[:n_ev]
    return seeds * (1.0 + np.diff(evo) / max(1, int(bins_per_event)))


def balance_events(costs, world: int) -> list[list[int]]:
    """Greedy balancing of whole events over `world` ranks by estimated cost:
    events in decreasing cost, each to the rank with the least total so far
    (ties to the lower rank); each rank's list comes back in event order."""
    if world < 1:
        raise ValueError("bad world")
    import heapq
    order = sorted(range(len(costs)), key=lambda e: (-float(costs[e]), e))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for e in order:
        tot, r = heapq.heappop(heap)
        out[r].append(e)
        heapq.heappush(heap, (tot + float(costs[e]), r))
    return [sorted(x) for x in out]


def combine(pg, units: float, step_ms: float, device=None):
    """(total units over ranks, slowest rank's step time) -- the job's throughput
    is total / slowest.  pg is torch.distributed (initialised) or None."""
    if pg is None:
        return float(units), float(step_ms)
    t = torch.tensor([float(units), float(step_ms)], dtype=torch.float64, device=device)
    u = t[:1].clone()
    m = t[1:].clone()
    pg.all_reduce(u, op=pg.ReduceOp.SUM)
    pg.all_reduce(m, op=pg.ReduceOp.MAX)
    return float(u.item()), float(m.item())
