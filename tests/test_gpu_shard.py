"""Sharding by whole events reproduces the unsharded result: the events of a
batch are balanced over three shards by estimated cost, each shard is binned and
found on its own (one after the other on one GPU, as separate ranks would), and
the per-shard outputs put back in seed order equal the output of one finding
call over all events bit for bit.  Seeds of different events never interact, so
the split is exact; this is what lets ranks run with no exchange on the data
path."""
import numpy as np
import pytest
import torch

from paper_1811_04141_gb300.shard import balance_events, event_costs
from synth import make_batch
from tests.gpu_helpers import make_ctx, to_np

pytestmark = pytest.mark.gpu


def _sub_batch(b, events):
    """Hits and seeds of the given events, hit indices renumbered from 0."""
    lo = b.event_offsets[:-1].astype(np.int64)
    hi = b.event_offsets[1:].astype(np.int64)
    hit_ids = np.concatenate([np.arange(lo[e], hi[e]) for e in events])
    new_of_old = np.full(b.n_hits, -1, dtype=np.int64)
    new_of_old[hit_ids] = np.arange(hit_ids.size)
    seeds = np.concatenate([np.nonzero(b.seed_event == e)[0] for e in events])
    evo = np.concatenate([[0], np.cumsum(hi[events] - lo[events])]).astype(np.int32)
    ev_new = np.zeros(b.n_events, dtype=np.int32)
    ev_new[events] = np.arange(len(events))
    return dict(xyz=b.xyz[:, hit_ids], layer=b.layer[hit_ids], evo=evo,
                sh=new_of_old[b.seed_hits[:, seeds]].astype(np.int32), se=ev_new[b.seed_event[seeds]],
                seeds=seeds, hit_ids=hit_ids)


def _find(ctx, xyz, layer, evo, sh, se, max_out):
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    bins = ctx.hits_bin(t(xyz, torch.float32), t(layer, torch.int32), t(evo, torch.int32))
    out = ctx.find(bins, t(sh, torch.int32), t(se, torch.int32), n_best=10, max_out=max_out)
    ctx.sync()
    return to_np(out)


def test_sequential_shards_reproduce_unsharded_output():
    b = make_batch("find20", list(range(7)), n_tracks=[150, 600, 300, 900, 200, 450, 700])
    ctx = make_ctx(b)
    max_out = len(b.layers) + 3
    full = _find(ctx, b.xyz, b.layer, b.event_offsets, b.seed_hits, b.seed_event, max_out)
    bins_per_event = sum(l["n_phi"] * l["n_zr"] for l in b.layers)
    shards = balance_events(event_costs(b.event_offsets, b.seed_event, bins_per_event), 3)
    assert sorted(sum(shards, [])) == list(range(b.n_events)) and all(shards)
    merged = {k: np.empty_like(v) for k, v in full.items()}
    for events in shards:
        s = _sub_batch(b, np.array(events))
        o = _find(ctx, s["xyz"], s["layer"], s["evo"], s["sh"], s["se"], max_out)
        for k, v in o.items():
            if k == "hits":
                v = np.where(v >= 0, s["hit_ids"][np.maximum(v, 0)], -1)
            merged[k][..., s["seeds"]] = v
    for k in full:
        a, m = full[k], merged[k]
        if a.dtype.kind == "f":
            assert np.array_equal(a.view(np.uint32), m.view(np.uint32)), k  # bit for bit, NaNs included
        else:
            assert np.array_equal(a, m), k
    ctx.close()
