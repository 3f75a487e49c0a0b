"""Persistent finding with per-event completion times, CUDA-graph replay of a
binning + finding step, and the block-size autotuner."""
import numpy as np
import pytest
import torch

from synth import make_batch
from tests.gpu_helpers import make_ctx, upload

pytestmark = pytest.mark.gpu


def test_graph_replay_equals_eager_and_event_times():
    from paper_1811_04141_gb300.runtime import CapturedStep
    rng = np.random.default_rng(5)
    n_ev = 12
    tracks = np.floor(np.exp(rng.uniform(np.log(50), np.log(800), n_ev))).astype(int)
    b = make_batch("dense45", list(range(200, 200 + n_ev)), n_tracks=list(tracks),
                   n_noise=list(np.floor(np.exp(rng.uniform(np.log(1e3), np.log(3e4), n_ev))).astype(int)))
    ctx = make_ctx(b)
    d = upload(b)
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    eager = ctx.find(bins, d["seed_hits"], d["seed_event"], n_best=10, max_out=48)
    ctx.sync()
    et = torch.zeros(n_ev + 1, dtype=torch.int64, device="cuda")
    step = CapturedStep(ctx, d["xyz"], d["layer"], d["event_offsets"], d["seed_hits"], d["seed_event"], n_best=10,
                        max_out=48, event_times=et)
    for _ in range(3):
        out = step.replay()
    torch.cuda.synchronize()
    assert torch.equal(out["hits"], eager["hits"]) and torch.equal(out["par"], eager["par"])
    t = et.cpu().numpy().astype(np.int64)
    lat = t[:n_ev] - t[n_ev]
    assert (lat > 0).all() and (lat < 10_000_000_000).all()


def test_autotuner_picks_a_valid_block_size():
    from paper_1811_04141_gb300.runtime import tune_find_block
    b = make_batch("find20", [61, 62], n_tracks=500)
    ctx = make_ctx(b)
    d = upload(b)
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    bt, rec = tune_find_block(ctx, bins, d["seed_hits"], d["seed_event"], n_best=10, cache=False, max_out=23)
    assert bt in (64, 128, 256) and len(rec["ms"]) == 3
    a = ctx.find(bins, d["seed_hits"], d["seed_event"], n_best=10, block_threads=bt, max_out=23)
    c = ctx.find(bins, d["seed_hits"], d["seed_event"], n_best=10, block_threads=128, max_out=23)
    ctx.sync()
    assert torch.equal(a["hits"], c["hits"]) and torch.equal(a["par"], c["par"])


def test_config_autotuner_grid_and_block():
    """The configuration tuner times every (bin grid, block size, seed order),
    loads the fastest grid, and the tracks found with its choice equal those of
    the default configuration bit for bit (the grid only accelerates the window
    search, the order only schedules the seeds)."""
    from paper_1811_04141_gb300.runtime import tune_find_config
    b = make_batch("dense45", [63, 64], n_tracks=800, n_noise=40000)
    ctx = make_ctx(b)
    d = upload(b)
    mo = len(b.layers) + 3
    ref_bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    ref = ctx.find(ref_bins, d["seed_hits"], d["seed_event"], n_best=10, max_out=mo)
    ctx.sync()
    ref = {k: v.clone() for k, v in ref.items() if v is not None}
    layers, bt, rec = tune_find_config(ctx, b.layers, b.bz, d["xyz"], d["layer"], d["event_offsets"],
                                       d["seed_hits"], d["seed_event"], n_best=10, cache=False, max_out=mo)
    assert len(rec["ms"]) == 16 and bt in (128, 256) and rec["seed_order"] in (0, 1) and rec["spread"] > 0
    assert all(l["n_phi"] == rec["grid"][0] and l["n_zr"] == rec["grid"][1] for l in layers)
    assert ctx.layers[0]["n_phi"] == rec["grid"][0]
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    out = ctx.find(bins, d["seed_hits"], d["seed_event"], n_best=10, block_threads=bt, max_out=mo,
                   seed_order=rec["seed_order"])
    ctx.sync()
    for k in ("hits", "n_hits", "status"):
        assert torch.equal(out[k], ref[k]), k
    for k in ("par", "cov", "chi2"):
        assert torch.equal(out[k].view(torch.int32), ref[k].view(torch.int32)), k
