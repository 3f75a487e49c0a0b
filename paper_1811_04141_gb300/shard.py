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
