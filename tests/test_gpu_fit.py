"""GPU fit (mkf_fit) against the FP64 oracle on the same FP32 hits."""
import numpy as np
import pytest
import torch

from synth import make_batch
from tests.gpu_helpers import (chi2_errors, chi2_ok, last_hits, make_ctx, oracle_fit, par_errors, steep_crossing, to_np,
                               upload)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg,tracks", [("fit10", 1000), ("fit10_b0", 1000), ("find20", 700), ("dense45", 500)])
def test_fit_parity(cfg, tracks):
    b = make_batch(cfg, [11], n_tracks=tracks)
    ctx = make_ctx(b)
    d = upload(b)
    out = to_np(ctx.fit(d["xyz"], d["layer"], d["track_hits"]))
    ctx.sync()
    ref = oracle_fit(b)
    assert (out["status"] == ref["status"]).all()
    assert (out["ndf"] == ref["ndf"]).all()
    ok = ref["status"] == 0
    e = par_errors(out["par"][:, ok], ref["par"][:, ok])
    assert e.max() <= 1.0, e.max(axis=1)
    c = chi2_errors(out["chi2"][ok], ref["chi2"][ok], ref["ndf"][ok])
    assert chi2_ok(out["chi2"][ok], ref["chi2"][ok], ref["ndf"][ok]), (np.quantile(c, 0.98), c.max())
    # covariance diagonal: relative 1e-3 (the prior shrinks by up to six orders
    # of magnitude over the seed hits, which the square-root form carries; up to
    # 2.3e-4 measured, 2e-2 with the covariance in FP32 entries through them)
    for i, k in enumerate((0, 2, 5, 9, 14, 20)):
        scale = np.maximum(np.abs(ref["cov"][k, ok]), 1e-9 * np.abs(ref["cov"][:, ok]).max(axis=0))
        r = np.abs(out["cov"][k, ok] - ref["cov"][k, ok]) / scale
        assert r.max() < 1e-3, (k, r.max())


def test_fit_given_seed_states_and_ragged_lists():
    """Caller-provided seeds, -1 gaps inside the hit lists, a ragged tail of
    tracks (n not a multiple of the block), and tracks with < 3 hits."""
    b = make_batch("find20", [12], n_tracks=333)
    hidx = b.track_hits.copy()
    hidx[4, ::3] = -1          # gaps
    hidx[3:, 7] = -1           # short track: 3 hits
    hidx[2:, 8] = -1           # too short: 2 hits -> bad seed
    ctx = make_ctx(b)
    d = upload(b)
    ht = torch.as_tensor(hidx, device="cuda")
    out = to_np(ctx.fit(d["xyz"], d["layer"], ht))
    ref = oracle_fit(b, hidx)
    assert out["status"][8] & 2 and ref["status"][8] & 2
    ok = ref["status"] == 0
    assert (out["status"] == ref["status"]).all()
    assert par_errors(out["par"][:, ok], ref["par"][:, ok]).max() <= 1.0
    # seeds given explicitly: the oracle's own seed state (FP32-rounded)
    import oracle as O
    geo = O.geometry_as_loaded(b)
    sp, sc = [], []
    for t in range(b.n_seeds):
        h = [x for x in hidx[:, t] if x >= 0][:3]
        if len(h) < 3:
            sp.append(np.zeros(6)); sc.append(np.eye(6))
            continue
        p, Cm = O.seed(geo, *[b.xyz[:, i].astype(np.float64) for i in h], b.layer[h[0]])
        sp.append(p); sc.append(Cm)
    sp = np.ascontiguousarray(np.array(sp).T, dtype=np.float32)
    sc = np.ascontiguousarray(O.pack21(np.array(sc)), dtype=np.float32)
    out2 = to_np(ctx.fit(d["xyz"], d["layer"], ht, torch.as_tensor(sp, device="cuda"),
                         torch.as_tensor(sc, device="cuda")))
    ref2 = O.fit(geo, b.xyz.astype(np.float64), b.layer, hidx, sp.astype(np.float64), sc.astype(np.float64))
    ok2 = ref2["status"] == 0
    assert par_errors(out2["par"][:, ok2], ref2["par"][:, ok2]).max() <= 1.0


def _backward_pair(b, hidx, inflate, ctx=None):
    """GPU and oracle backward fits from the same start: the oracle's forward fit
    at the last hit, rounded to FP32, given to both."""
    import oracle as O
    geo = O.geometry_as_loaded(b)
    f = O.fit(geo, b.xyz.astype(np.float64), b.layer, hidx)
    lp = np.ascontiguousarray(f["par"], dtype=np.float32)
    lc = np.ascontiguousarray(f["cov"], dtype=np.float32)
    ctx = ctx or make_ctx(b)
    d = upload(b)
    out = to_np(ctx.fit_backward(d["xyz"], d["layer"], torch.as_tensor(hidx, device="cuda"),
                                 torch.as_tensor(lp, device="cuda"), torch.as_tensor(lc, device="cuda"), inflate))
    ctx.sync()
    ref = O.fit_backward(geo, b.xyz.astype(np.float64), b.layer, hidx, lp.astype(np.float64), lc.astype(np.float64),
                         inflate)
    return out, ref, f


@pytest.mark.parametrize("cfg,tracks,inflate", [("fit10", 1000, 100.0), ("fit10_b0", 1000, 100.0),
                                                ("find20", 700, 100.0), ("dense45", 500, 1e4),
                                                ("find20", 300, 1.0)])
def test_fit_backward_parity(cfg, tracks, inflate):
    """Backward fit (mkf_fit_backward) against the oracle's backward pass: state
    at the first hit, chi2, ndf, status and covariance diagonal."""
    b = make_batch(cfg, [14], n_tracks=tracks)
    out, ref, f = _backward_pair(b, b.track_hits, inflate)
    assert (out["status"] == ref["status"]).all()
    assert (out["ndf"] == ref["ndf"]).all()
    ok = (ref["status"] == 0) & (f["status"] == 0)
    assert ok.mean() > 0.95
    e = par_errors(out["par"][:, ok], ref["par"][:, ok], ref["cov"][:, ok])
    assert e.max() <= 1.0, e.max(axis=1)
    c = chi2_errors(out["chi2"][ok], ref["chi2"][ok], ref["ndf"][ok])
    assert chi2_ok(out["chi2"][ok], ref["chi2"][ok], ref["ndf"][ok]), (np.quantile(c, 0.98), c.max())
    # the start inflated 1e4 shrinks by as much over the first hits (9.5e-3
    # measured there, up to 2.4e-4 at inflation 1-100)
    bar = 2e-2 if inflate > 100.0 else 1e-3
    for k in (0, 2, 5, 9, 14, 20):
        scale = np.maximum(np.abs(ref["cov"][k, ok]), 1e-9 * np.abs(ref["cov"][:, ok]).max(axis=0))
        r = np.abs(out["cov"][k, ok] - ref["cov"][k, ok]) / scale
        assert r.max() < bar, (k, r.max())


def test_fit_backward_ragged_lists_and_errors():
    """-1 gaps inside the lists, a 3-hit track, a 2-hit track (no fit), a ragged
    tail of tracks; argument errors."""
    b = make_batch("find20", [15], n_tracks=333)
    hidx = b.track_hits.copy()
    hidx[4, ::3] = -1
    hidx[3:, 7] = -1
    hidx[2:, 8] = -1
    out, ref, f = _backward_pair(b, hidx, 100.0)
    assert out["status"][8] & 2 and ref["status"][8] & 2 and np.isnan(out["par"][:, 8]).all()
    assert (out["status"] == ref["status"]).all()
    ok = (ref["status"] == 0) & (f["status"] == 0)
    assert par_errors(out["par"][:, ok], ref["par"][:, ok], ref["cov"][:, ok]).max() <= 1.0
    from paper_1811_04141_gb300._native import MkfError
    ctx = make_ctx(b)
    d = upload(b)
    lp = torch.zeros(6, b.n_seeds, device="cuda")
    lc = torch.zeros(21, b.n_seeds, device="cuda")
    for bad in (0.5, float("nan"), float("inf")):
        with pytest.raises(MkfError):
            ctx.fit_backward(d["xyz"], d["layer"], d["track_hits"], lp, lc, bad)
    empty = torch.empty(10, 0, dtype=torch.int32, device="cuda")
    o = ctx.fit_backward(d["xyz"], d["layer"], empty, lp[:, :0].contiguous(), lc[:, :0].contiguous(), 100.0)
    assert o["par"].shape == (6, 0)


@pytest.mark.parametrize("cfg,material,eloss", [("fit10", 0.03, 0.0), ("fit10", 0.03, 0.15), ("fit10_b0", 0.02, 0.0)])
def test_fit_with_material_parity(cfg, material, eloss):
    """Forward and backward fit with material (tracks scattered by the
    generator in `material` X0 per layer, losing energy when eloss > 0) against
    the oracle."""
    b = make_batch(cfg, [16], n_tracks=800, material=material, eloss=eloss)
    assert all(d["x0"] == material for d in b.layers)
    ctx = make_ctx(b)
    d = upload(b)
    out = to_np(ctx.fit(d["xyz"], d["layer"], d["track_hits"]))
    ctx.sync()
    ref = oracle_fit(b)
    assert (out["status"] == ref["status"]).all()
    ok = ref["status"] == 0
    assert par_errors(out["par"][:, ok], ref["par"][:, ok], ref["cov"][:, ok]).max() <= 1.0
    assert chi2_ok(out["chi2"][ok], ref["chi2"][ok], ref["ndf"][ok])
    # covariance diagonal: with scattering noise the FP32 filter's covariance
    # loses more to conditioning (each update shrinks a prior widened by the
    # noise) than without it: 99 % of the tracks within 5e-3 relative on each
    # variance, every track crossing its last layer steeply within 3e-2
    # (steep_crossing; measured 2.2e-3 and 1.3e-2); x and y against the
    # transverse position variance (on a cylinder one of them is nearly
    # radial, with a variance close to zero)
    pos = ref["cov"][0, ok] + ref["cov"][2, ok]
    steep = steep_crossing(b, last_hits(b)[ok])
    for k in (0, 2, 5, 9, 14, 20):
        floor = 1e-2 * pos if k in (0, 2) else 1e-9 * np.abs(ref["cov"][:, ok]).max(axis=0)
        r = np.abs(out["cov"][k, ok] - ref["cov"][k, ok]) / np.maximum(np.abs(ref["cov"][k, ok]), floor)
        assert np.quantile(r, 0.99) < 5e-3 and r[steep].max() < 3e-2, (k, np.quantile(r, 0.99), r[steep].max())
    outb, refb, f = _backward_pair(b, b.track_hits, 100.0, ctx)
    okb = (refb["status"] == 0) & (f["status"] == 0)
    assert (outb["status"] == refb["status"]).all()
    assert par_errors(outb["par"][:, okb], refb["par"][:, okb], refb["cov"][:, okb]).max() <= 1.0
    assert chi2_ok(outb["chi2"][okb], refb["chi2"][okb], refb["ndf"][okb])


@pytest.mark.parametrize("cfg,alpha", [("fit10", 1e-5), ("find20", 1e-6)])
def test_fit_in_parameterised_field_parity(cfg, alpha):
    """Forward and backward fit in the parameterised field (the Runge-Kutta
    variant) against the oracle, on tracks the generator moves through that
    field (find20: disks up to z = 270 cm)."""
    b = make_batch(cfg, [17], n_tracks=800 if cfg == "fit10" else 500, field_alpha=alpha)
    ctx = make_ctx(b)
    d = upload(b)
    out = to_np(ctx.fit(d["xyz"], d["layer"], d["track_hits"]))
    ctx.sync()
    ref = oracle_fit(b)
    assert (out["status"] == ref["status"]).all()
    ok = ref["status"] == 0
    assert par_errors(out["par"][:, ok], ref["par"][:, ok], ref["cov"][:, ok]).max() <= 1.0
    assert chi2_ok(out["chi2"][ok], ref["chi2"][ok], ref["ndf"][ok])
    # covariance diagonal without material: every track within 1e-3 (5.8e-5 measured)
    pos = ref["cov"][0, ok] + ref["cov"][2, ok]
    for k in (0, 2, 5, 9, 14, 20):
        floor = 1e-2 * pos if k in (0, 2) else 1e-9 * np.abs(ref["cov"][:, ok]).max(axis=0)
        r = np.abs(out["cov"][k, ok] - ref["cov"][k, ok]) / np.maximum(np.abs(ref["cov"][k, ok]), floor)
        assert r.max() < 1e-3, (k, r.max())
    outb, refb, f = _backward_pair(b, b.track_hits, 100.0, ctx)
    okb = (refb["status"] == 0) & (f["status"] == 0)
    assert (outb["status"] == refb["status"]).all()
    assert par_errors(outb["par"][:, okb], refb["par"][:, okb], refb["cov"][:, okb]).max() <= 1.0
    assert chi2_ok(outb["chi2"][okb], refb["chi2"][okb], refb["ndf"][okb])


def test_fit_with_material_map_parity():
    """Forward and backward fit with an r-z material map (each crossing's
    scattering and energy loss from its cell) on tracks the generator scatters
    and slows with the same map, against the oracle."""
    from tests.test_oracle_material_map import _graded_map
    b = make_batch("fit10", [18], n_tracks=800, material_map=_graded_map())
    ctx = make_ctx(b)
    d = upload(b)
    out = to_np(ctx.fit(d["xyz"], d["layer"], d["track_hits"]))
    ctx.sync()
    ref = oracle_fit(b)
    assert (out["status"] == ref["status"]).all()
    ok = ref["status"] == 0
    assert par_errors(out["par"][:, ok], ref["par"][:, ok], ref["cov"][:, ok]).max() <= 1.0
    assert chi2_ok(out["chi2"][ok], ref["chi2"][ok], ref["ndf"][ok])
    outb, refb, f = _backward_pair(b, b.track_hits, 100.0, ctx)
    okb = (refb["status"] == 0) & (f["status"] == 0)
    assert (outb["status"] == refb["status"]).all()
    assert par_errors(outb["par"][:, okb], refb["par"][:, okb], refb["cov"][:, okb]).max() <= 1.0
    assert chi2_ok(outb["chi2"][okb], refb["chi2"][okb], refb["ndf"][okb])


@pytest.mark.parametrize("cfg,kw", [("fit10", {}), ("find20", {}), ("fit10", dict(material=0.03, eloss=0.04)),
                                    ("fit10", dict(field_alpha=1e-5))])
def test_fit_smooth_parity(cfg, kw):
    """Smoothed states at every hit (mkf_fit_smooth, inflate 100) against the
    oracle's smoother: parameters at every hit, the covariance diagonal as in
    the fit tests with material (its maximum where the track does not graze the
    layer), chi2 and status of the forward pass."""
    import oracle as O
    b = make_batch(cfg, [19], n_tracks=600, **kw)
    ctx = make_ctx(b)
    d = upload(b)
    out = to_np(ctx.fit_smooth(d["xyz"], d["layer"], d["track_hits"], inflate=100.0))
    ctx.sync()
    ref = O.fit_smooth(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.track_hits, inflate=100.0)
    # An FP32 update cannot resolve a posterior 2^20 times narrower than its
    # prior (fewer than 4 of the 24 bits are left): the backward filter starts
    # from the inflated forward state, and with material (its scattering makes
    # the angles at the last hit poorly known) a low-pT track can reach its next
    # hit with a prior ~1e7 times the hit's variance.  Only where the oracle
    # logged such an update may the GPU flag the non-positive-definite residual
    # covariance it meets after it (MKF_ST_BADS); those tracks are left out below.
    diff = out["status"] != ref["status"]
    assert (ref["shrink"][diff] >= 2.0 ** 20).all(), ref["shrink"][diff]
    assert ((out["status"][diff] & ~np.uint32(O.ST_BADS)) == ref["status"][diff]).all()
    assert diff.mean() <= 0.005
    ok = (ref["status"] == 0) & ~diff
    assert chi2_ok(out["chi2"][ok], ref["chi2"][ok], ref["ndf"][ok])
    m = (b.track_hits >= 0) & ok[None, :]
    assert np.array_equal(np.isnan(out["par"][:, 0]) & m, np.isnan(ref["par"][:, 0]) & m)
    gp, rp = np.transpose(out["par"], (1, 0, 2))[:, m], np.transpose(ref["par"], (1, 0, 2))[:, m]
    gc, rc = np.transpose(out["cov"], (1, 0, 2))[:, m], np.transpose(ref["cov"], (1, 0, 2))[:, m]
    assert par_errors(gp, rp, rc).max() <= 1.0
    steep = steep_crossing(b, b.track_hits[m])
    pos = rc[0] + rc[2]
    for k in (0, 2, 5, 9, 14, 20):
        floor = 1e-2 * pos if k in (0, 2) else 1e-9 * np.abs(rc).max(axis=0)
        r = np.abs(gc[k] - rc[k]) / np.maximum(np.abs(rc[k]), floor)
        assert np.quantile(r, 0.99) < 5e-2 and r[steep].max() < 1.5e-1, (k, np.quantile(r, 0.99))


def test_fit_empty_and_errors():
    b = make_batch("fit10", [13], n_tracks=10)
    ctx = make_ctx(b)
    d = upload(b)
    empty = torch.empty(10, 0, dtype=torch.int32, device="cuda")
    out = ctx.fit(d["xyz"], d["layer"], empty)
    assert out["par"].shape == (6, 0)
    from paper_1811_04141_gb300._native import MkfError
    with pytest.raises(MkfError):
        ctx.fit(d["xyz"], d["layer"], torch.zeros(65, 4, dtype=torch.int32, device="cuda"))


def test_fit_full_size_sampled():
    """The 10^6-track fit workload (as timed by the bench), checked on a sample of
    tracks against the oracle."""
    from tests.gpu_helpers import O
    b = make_batch("fit10", list(range(1000)))
    ctx = make_ctx(b)
    d = upload(b)
    out = to_np(ctx.fit(d["xyz"], d["layer"], d["track_hits"]))
    ctx.sync()
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(b.n_seeds, 2000, replace=False))
    ref = oracle_fit(b, np.ascontiguousarray(b.track_hits[:, sel]))
    ok = ref["status"] == 0
    assert par_errors(out["par"][:, sel][:, ok], ref["par"][:, ok]).max() <= 1.0
    assert chi2_ok(out["chi2"][sel][ok], ref["chi2"][ok], ref["ndf"][ok])
    assert np.isfinite(out["par"]).all()
