"""Parity at the full sizes of the dense and batched finding workloads, in the
launch configurations the bench times, on seeds sampled across all events
(the oracle scans every hit of a layer, so it takes a sample)."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import make_batch
from tests.gpu_helpers import compare, make_ctx, to_np, upload

pytestmark = pytest.mark.gpu


def _oracle(b, sel, n_best=10):
    return O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                  n_best=n_best, seed_list=sel, max_out=len(b.layers) + 3)


def test_dense_50_events_sampled():
    """50 events x 6000 tracks (pT^-3) + 200k noise hits each, 17 cylinders +
    2 x 14 disks, N = 10, with the bin grid, block size and seed order the
    tuner picks for it (as the bench's dense leg runs it)."""
    from paper_1811_04141_gb300.runtime import tune_find_config
    b = make_batch("dense45", list(range(300, 350)))
    ctx = make_ctx(b)
    d = upload(b)
    mo = len(b.layers) + 3
    _, bt, rec = tune_find_config(ctx, b.layers, b.bz, d["xyz"], d["layer"], d["event_offsets"], d["seed_hits"],
                                  d["seed_event"], n_best=10, cache=False, max_out=mo)
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    out = to_np(ctx.find(bins, d["seed_hits"], d["seed_event"], n_best=10, max_out=mo, block_threads=bt,
                         seed_order=rec["seed_order"]))
    ctx.sync()
    sel = np.sort(np.random.default_rng(3).choice(b.n_seeds, 150, replace=False))
    compare(out, _oracle(b, sel), sel)
    assert (out["n_hits"] >= 3).all() and np.isfinite(out["par"]).all()


def test_batched_512_uneven_events_graph_replay_sampled():
    """512 events with log-uniform track (100-20000) and noise (1e3-3e5) counts,
    one binning + finding step captured in a CUDA graph with the autotuned bin
    grid, block size and seed order and replayed, as the bench's headline runs
    it."""
    from paper_1811_04141_gb300.runtime import CapturedStep, tune_find_config
    rng = np.random.default_rng(4_181_104)
    n_ev = 512
    tracks = np.floor(np.exp(rng.uniform(np.log(100), np.log(20000), n_ev))).astype(int)
    noise = np.floor(np.exp(rng.uniform(np.log(1e3), np.log(3e5), n_ev))).astype(int)
    b = make_batch("dense45", list(range(5000, 5000 + n_ev)), n_tracks=list(tracks), n_noise=list(noise))
    ctx = make_ctx(b)
    d = upload(b)
    mo = len(b.layers) + 3
    _, bt, rec = tune_find_config(ctx, b.layers, b.bz, d["xyz"], d["layer"], d["event_offsets"], d["seed_hits"],
                                  d["seed_event"], n_best=10, cache=False, max_out=mo)
    et = torch.zeros(n_ev + 1, dtype=torch.int64, device="cuda")
    step = CapturedStep(ctx, d["xyz"], d["layer"], d["event_offsets"], d["seed_hits"], d["seed_event"], n_best=10,
                        max_out=mo, block_threads=bt, seed_order=rec["seed_order"], event_times=et)
    for _ in range(2):
        out = step.replay()
    torch.cuda.synchronize()
    out = to_np(out)
    # seeds sampled evenly over the events (small and large ones alike)
    ev_of_seed = b.seed_event
    rs = np.random.default_rng(9)
    sel = np.sort(np.concatenate([rs.choice(np.nonzero(ev_of_seed == e)[0], 1) for e in rs.choice(n_ev, 160, replace=False)
                                  if (ev_of_seed == e).any()]))
    compare(out, _oracle(b, sel), sel)
    t = et.cpu().numpy().astype(np.int64)
    assert (t[:n_ev] > t[n_ev]).all()  # every event completed after the launch started
