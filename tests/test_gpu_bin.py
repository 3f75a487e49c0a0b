"""GPU hit binning (mkf_hits_bin): exact integer properties of the counting sort."""
import numpy as np
import pytest
import torch

from synth import make_batch
from tests.gpu_helpers import make_ctx, upload

pytestmark = pytest.mark.gpu


def _layer_bases(layers):
    base, out = 0, []
    for d in layers:
        out.append(base)
        base += d["n_phi"] * d["n_zr"]
    return np.array(out), base


@pytest.mark.parametrize("cfg,events,tracks,grid", [
    ("find20", 3, 500, None),
    ("dense45", 2, 800, None),
    # hundreds of scan tiles (each tile adds the totals of the tiles before it)
    ("dense45", 12, 50, None),
    # two bins per layer: a block's 256 bins hold more hits than its shared buffer,
    # so the in-bin ordering runs in global memory
    ("find20", 3, 300, (2, 1)),
])
def test_binning_is_a_permutation_into_the_right_bins(cfg, events, tracks, grid):
    b = make_batch(cfg, list(range(events)), n_tracks=tracks)
    if grid is not None:
        b.layers = [dict(d, n_phi=grid[0], n_zr=grid[1]) for d in b.layers]
    ctx = make_ctx(b)
    d = upload(b)
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    ctx.sync()
    ex = bins.export(ctx)
    torch.cuda.synchronize()
    rec, inv, off = ex["rec"].cpu().numpy(), ex["inv"].cpu().numpy(), ex["offsets"].cpu().numpy()
    bases, per_event = _layer_bases(b.layers)
    assert ex["n_bins"] == per_event * b.n_events
    # CSR offsets: monotone, cover every hit
    assert off[0] == 0 and off[-1] == b.n_hits and (np.diff(off) >= 0).all()
    orig = rec[:, 3].view(np.int32)
    # a permutation, inverse consistent
    assert np.array_equal(np.sort(orig), np.arange(b.n_hits))
    assert np.array_equal(inv[orig], np.arange(b.n_hits))
    # coordinates copied exactly (z on cylinders, r on disks in the third slot)
    kinds = np.array([l["kind"] for l in b.layers])
    assert np.array_equal(rec[:, 0], b.xyz[0, orig]) and np.array_equal(rec[:, 1], b.xyz[1, orig])
    cyl = kinds[b.layer[orig]] == 0
    assert np.array_equal(rec[cyl, 2], b.xyz[2, orig[cyl]])
    # every hit sits in its own (event, layer) block and ascending original index within a bin
    bin_of = np.repeat(np.arange(off.size - 1), np.diff(off))
    ev_of = np.searchsorted(b.event_offsets, orig, side="right") - 1
    lay = b.layer[orig]
    local = bin_of - ev_of * per_event - bases[lay]
    nphi = np.array([l["n_phi"] for l in b.layers])[lay]
    nzr = np.array([l["n_zr"] for l in b.layers])[lay]
    assert (local >= 0).all() and (local < nphi * nzr).all()
    same = bin_of[1:] == bin_of[:-1]
    assert (orig[1:][same] > orig[:-1][same]).all()
    # phi and z/r bins agree with a float64 recomputation except within rounding of an edge
    phi = np.arctan2(b.xyz[1, orig].astype(np.float64), b.xyz[0, orig].astype(np.float64))
    fpb = (phi + np.pi) * nphi / (2 * np.pi)
    pb = local // nzr
    assert (np.abs(np.clip(np.floor(fpb), 0, nphi - 1) - pb) == 0)[np.abs(fpb - np.round(fpb)) > 1e-4].all()


def test_binning_reuse_and_empty():
    b = make_batch("find20", [5], n_tracks=200)
    ctx = make_ctx(b)
    d = upload(b)
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    # refill the same store with a smaller input
    b2 = make_batch("find20", [6], n_tracks=50)
    d2 = upload(b2)
    bins = ctx.hits_bin(d2["xyz"], d2["layer"], d2["event_offsets"], bins)
    ex = bins.export(ctx)
    torch.cuda.synchronize()
    assert ex["n_hits"] == b2.n_hits and ex["offsets"][-1].item() == b2.n_hits
    # more events (more bins than any call before), fewer, then as many again: the
    # histogram left by each call must be zero for the next (a count left over
    # would show as a gap in the offsets)
    b3 = make_batch("find20", [7, 8, 9], n_tracks=120)
    d3 = upload(b3)
    for bb, dd in ((b3, d3), (b2, d2), (b3, d3), (b, d)):
        bins = ctx.hits_bin(dd["xyz"], dd["layer"], dd["event_offsets"], bins)
        ex = bins.export(ctx)
        torch.cuda.synchronize()
        off = ex["offsets"].cpu().numpy()
        orig = ex["rec"].cpu().numpy()[:, 3].view(np.int32)
        assert off[0] == 0 and off[-1] == bb.n_hits and (np.diff(off) >= 0).all()
        assert np.array_equal(np.sort(orig), np.arange(bb.n_hits))
    # an event with no hits at all
    empty_xyz = torch.zeros(3, 0, device="cuda")
    e = ctx.hits_bin(empty_xyz, torch.zeros(0, dtype=torch.int32, device="cuda"),
                     torch.zeros(2, dtype=torch.int32, device="cuda"))
    assert e.info()["n_hits"] == 0
    ctx.sync()


def test_binning_flags_bad_layer_ids():
    from paper_1811_04141_gb300._native import MkfError
    b = make_batch("find20", [7], n_tracks=50)
    ctx = make_ctx(b)
    d = upload(b)
    bad = d["layer"].clone()
    bad[5] = 99
    ctx.hits_bin(d["xyz"], bad, d["event_offsets"])
    with pytest.raises(MkfError):
        ctx.sync()
    ctx.sync()  # the record is cleared after being reported
