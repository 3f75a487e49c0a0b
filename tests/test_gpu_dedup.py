"""GPU seed cleaning (mkf_seeds_clean) and duplicate-track removal
(mkf_tracks_dedup) against the oracle: keep flags bit-exact on the same inputs."""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.dedup as D
from synth import make_batch
from tests.gpu_helpers import make_ctx, upload

pytestmark = pytest.mark.gpu


def _t(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("cfg,tracks", [("find20", 1500), ("dense45", 1200)])
def test_seeds_clean_parity(cfg, tracks):
    b = make_batch(cfg, [0, 1], n_tracks=tracks, overlap=0.1)
    geo = O.geometry_as_loaded(b)
    par = O.fit(geo, b.xyz.astype(np.float64), b.layer, b.seed_hits)["par"].astype(np.float32)
    ctx = make_ctx(b)
    for tol in ((0.15, 0.02, 0.02), (5.0, 3.0, 4.0), (0.0, 0.0, 0.0), (0.05, 0.002, 0.002)):
        keep = ctx.seeds_clean(_t(b.seed_hits, torch.int32), b.n_hits, _t(par, torch.float32), *tol)
        ctx.sync()
        ref = D.clean_seeds(b.seed_hits, b.n_hits, par, *tol)
        assert (keep.cpu().numpy().astype(bool) == ref).all(), tol
    # the default tolerances remove exactly the repeated seeds here
    keep = ctx.seeds_clean(_t(b.seed_hits, torch.int32), b.n_hits, _t(par, torch.float32)).cpu().numpy()
    assert (keep.astype(bool) == (b.seed_dup_of < 0)).all()


def test_tracks_dedup_parity_after_oracle_finding():
    b = make_batch("find20", [3], n_tracks=400, overlap=0.15)
    geo = O.geometry_as_loaded(b)
    r = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=10,
               max_out=len(b.layers) + 3)
    c2 = r["chi2"].astype(np.float32)
    ctx = make_ctx(b)
    for f in (0.5, 0.0, 0.3, 1.0):
        keep = ctx.tracks_dedup(_t(r["hits"], torch.int32), b.n_hits, _t(r["n_hits"], torch.int32),
                                _t(c2, torch.float32), f)
        ctx.sync()
        ref = D.dedup_tracks(r["hits"], b.n_hits, r["n_hits"], c2, f)
        assert (keep.cpu().numpy().astype(bool) == ref).all(), f


@pytest.mark.parametrize("seed", range(3))
def test_dedup_parity_random_lists(seed):
    """Random lists: repeated hits inside a list, indices outside [0, n_hits),
    many exact chi2 ties, a ragged tail of items."""
    rng = np.random.default_rng(seed)
    n, n_hits = 3001, 900
    b = make_batch("fit10", [0], n_tracks=5)
    ctx = make_ctx(b)
    sh = rng.integers(-3, n_hits + 5, size=(3, n)).astype(np.int32)
    par = np.zeros((6, n), np.float32)
    par[3] = rng.choice([-1.0, 1.0], n) * rng.uniform(0.1, 0.3, n)
    par[4] = rng.uniform(-np.pi, np.pi, n)
    par[5] = rng.uniform(0.2, 2.9, n)
    keep = ctx.seeds_clean(_t(sh, torch.int32), n_hits, _t(par, torch.float32), 0.1, 1.0, 1.5).cpu().numpy()
    assert (keep.astype(bool) == D.clean_seeds(sh, n_hits, par, 0.1, 1.0, 1.5)).all()
    hidx = rng.integers(-2, n_hits + 2, size=(12, n)).astype(np.int32)
    hidx[3] = hidx[1]  # a hit listed twice
    nh = rng.integers(3, 13, n).astype(np.int32)
    c2 = rng.integers(0, 3, n).astype(np.float32)
    for f in (0.0, 0.25, 0.5, 1.0):
        keep = ctx.tracks_dedup(_t(hidx, torch.int32), n_hits, _t(nh, torch.int32), _t(c2, torch.float32), f)
        assert (keep.cpu().numpy().astype(bool) == D.dedup_tracks(hidx, n_hits, nh, c2, f)).all(), f


def test_gpu_pipeline_removes_duplicates():
    """GPU finding from every seed of overlap events, then GPU removal: one track
    per particle, no particle lost (properties only)."""
    b = make_batch("find20", [4], n_tracks=600, overlap=0.15)
    ctx = make_ctx(b)
    d = upload(b)
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    out = ctx.find(bins, d["seed_hits"], d["seed_event"], n_best=10, max_out=len(b.layers) + 3)
    keep = ctx.tracks_dedup(out["hits"], b.n_hits, out["n_hits"], out["chi2"]).cpu().numpy().astype(bool)
    ctx.sync()
    hits = out["hits"].cpu().numpy()
    owner = np.where(hits >= 0, b.hit_particle[np.maximum(hits, 0)], -2)
    frac = (owner == b.seed_particle[None, :]).sum(0) / np.maximum((hits >= 0).sum(0), 1)
    matched = frac >= 0.75
    assert set(b.seed_particle[matched & keep]) == set(b.seed_particle[matched])
    assert np.bincount(b.seed_particle[matched & keep]).max() == 1


def test_dedup_empty_and_errors():
    b = make_batch("fit10", [0], n_tracks=5)
    ctx = make_ctx(b)
    from paper_1811_04141_gb300._native import MkfError
    z3 = torch.empty(3, 0, dtype=torch.int32, device="cuda")
    assert ctx.seeds_clean(z3, 10, torch.empty(6, 0, device="cuda")).shape == (0,)
    zh = torch.empty(5, 0, dtype=torch.int32, device="cuda")
    assert ctx.tracks_dedup(zh, 10, torch.empty(0, dtype=torch.int32, device="cuda"),
                            torch.empty(0, device="cuda")).shape == (0,)
    sh = torch.zeros(3, 4, dtype=torch.int32, device="cuda")
    par = torch.zeros(6, 4, device="cuda")
    with pytest.raises(MkfError):
        ctx.seeds_clean(sh, 10, par, -1.0)
    hi = torch.zeros(5, 4, dtype=torch.int32, device="cuda")
    with pytest.raises(MkfError):
        ctx.tracks_dedup(hi, 10, torch.ones(4, dtype=torch.int32, device="cuda"), torch.zeros(4, device="cuda"), 1.5)
    # no valid hits: everything kept
    keep = ctx.tracks_dedup(hi, 0, torch.ones(4, dtype=torch.int32, device="cuda"), torch.zeros(4, device="cuda"))
    assert (keep.cpu().numpy() == 1).all()
