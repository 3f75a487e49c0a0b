"""Learned pruning on the GPU: the finder's feature dump and its MLP-pruned
branching against the FP64 oracle (same bfloat16 weights, same threshold), and
an end-to-end training run whose gain over the plain finder is measured."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp
from synth import make_batch
from tests.gpu_helpers import make_ctx, to_np, upload

pytestmark = pytest.mark.gpu

TIE_MLP = 2e-2   # |logit - tau| below which FP32 and FP64 may decide differently
TIE_SCORE, TIE_CUT, TIE_GEO = 5e-3, 2e-3, 1e-4


def _gpu(ctx, b, **kw):
    d = upload(b)
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    out = ctx.find(bins, d["seed_hits"], d["seed_event"], max_out=len(b.layers) + 3, **kw)
    ctx.sync()
    return out, d


def test_feature_dump_matches_oracle():
    """N = 1: one candidate per seed, so (seed, hit) names a pair uniquely."""
    from paper_1811_04141_gb300.api import feature_buffer
    b = make_batch("dense45", [51], n_tracks=600, n_noise=40000)
    ctx = make_ctx(b)
    fb = feature_buffer(200000)
    _gpu(ctx, b, n_best=1, feat=fb)
    m = int(fb["count"].item())
    g_feat, g_ref = fb["feat"][:m].cpu().numpy(), fb["ref"][:m].cpu().numpy()
    r = O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
               n_best=1, dump_cap=200000)
    o_feat, o_ref = r["feat"], r["feat_ref"]
    gk = {(int(s), int(h)): i for i, (s, h, _) in enumerate(g_ref)}
    ok = [(gk[(int(s), int(h))], i) for i, (s, h, _) in enumerate(o_ref) if (int(s), int(h)) in gk]
    assert len(ok) >= 0.995 * len(o_ref) and len(o_ref) > 1000
    gi, oi = np.array(ok).T
    d = np.abs(g_feat[gi] - o_feat[oi])
    # residual pulls and chi2 carry the FP32 precision of the residuals (~1e-3 of a
    # resolution, see the fit tolerances); counts and flags are exact
    tol = np.array([1e-2, 1e-2, 1e-4, 1e-3, 1e-6, 1e-6, 1e-6, 0, 1e-5, 1e-5, 1e-4, 1e-4])
    rel = np.array([0, 0, 1e-2, 1e-2, 0, 0, 0, 0, 1e-4, 1e-4, 1e-3, 1e-3]) * np.abs(o_feat[oi])
    assert (d <= tol + rel).mean(axis=0).min() >= 0.999, (d / (tol + rel + 1e-30)).max(axis=0)
    assert (g_ref[gi, 2] == o_ref[oi, 2]).mean() >= 0.999


@pytest.mark.parametrize("tau", [-1.0, 0.5])
def test_pruned_find_matches_oracle(tau):
    b = make_batch("dense45", [52], n_tracks=500, n_noise=60000)
    ctx = make_ctx(b)
    w = mlp.init_weights(21)
    from paper_1811_04141_gb300.api import mkf_mlp_to_bf16
    wb = mkf_mlp_to_bf16(ctx, torch.as_tensor(w, device="cuda"))
    out, _ = _gpu(ctx, b, n_best=10, mlp_bf16=wb, mlp_tau=tau)
    out = to_np(out)
    ref = O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                 n_best=10, mlp_w=mlp.bf16_round(w), mlp_tau=tau, max_out=len(b.layers) + 3)
    same = (out["hits"] == ref["hits"]).all(axis=0)
    m = ref["margins"]
    for k in np.nonzero(~same)[0]:
        assert m[0, k] < TIE_SCORE or m[1, k] < TIE_CUT or m[2, k] < TIE_GEO or m[3, k] < TIE_MLP, (k, m[:, k])
    assert same.mean() >= 0.999
    # the MLP did prune something at these thresholds
    plain = O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                   n_best=10, max_out=len(b.layers) + 3)
    assert ref["counters"][2].sum() != plain["counters"][2].sum() or np.isfinite(m[3]).any()


def test_training_and_gain_over_plain_finder():
    """Train on features the plain finder dumps (labels from truth), choose the
    largest threshold keeping efficiency within 0.5 points of the plain finder
    on the training events, and measure on held-out events: efficiency within
    0.5 points, and the work saved (candidate-layers, updates)."""
    from paper_1811_04141_gb300 import learned as L
    tr = make_batch("dense45", [1001, 1002, 1003], n_tracks=3000, n_noise=100000)
    ev = make_batch("dense45", [11, 12], n_tracks=3000, n_noise=100000)
    ctx = make_ctx(tr)

    def prep(b):
        d = upload(b)
        d["bins"] = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
        d["hp"] = torch.as_tensor(b.hit_particle, device="cuda")
        d["sp"] = torch.as_tensor(b.seed_particle, device="cuda")
        return d

    dt, de = prep(tr), prep(ev)
    feat, ref = L.collect_features(ctx, dt["bins"], dt["seed_hits"], dt["seed_event"], 4_000_000, n_best=10)
    lab = L.label_pairs(ref, dt["hp"], dt["sp"])
    st = L.train(ctx, feat, lab, steps=800, batch=4096, lr=2e-3)
    assert st["losses"][-1] < st["losses"][0]

    def run(d, tau=None):
        kw = dict(n_best=10)
        if tau is not None:
            kw.update(mlp_bf16=st["w_bf16"], mlp_tau=tau)
        out = ctx.find(d["bins"], d["seed_hits"], d["seed_event"], **kw)
        ctx.sync()
        e, f = L.efficiency(out["hits"], d["hp"], d["sp"])
        return e, f, out["counters"].sum(dim=1).cpu().numpy()

    e0, f0, c0 = run(dt)
    best = L.choose_tau(lambda t: run(dt, t)[:2], e0, [-4, -2, -1, 0, 1, 2])
    assert best is not None
    tau = best[0]
    ep, fp, cp = run(de)
    el, fl, cl = run(de, tau)
    print(f"learned pruning: tau={tau} eff {ep:.4f}->{el:.4f} fake {fp:.4f}->{fl:.4f} "
          f"cand-layers {cp[0]}->{cl[0]} updates {cp[2]}->{cl[2]}")
    assert el >= ep - 0.005 and fl <= fp + 0.005
    assert cl[0] <= cp[0] and cl[2] <= cp[2]
