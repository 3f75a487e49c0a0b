"""Learned pruning on the GPU: the finder's feature dump and its MLP-pruned
branching against the FP64 oracle (same bfloat16 weights, same threshold), and
an end-to-end training run whose gain over the plain finder is measured."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp
from synth import make_batch
from tests.gpu_helpers import TIE_CUT, TIE_GEO, TIE_SCORE, make_ctx, to_np, upload

pytestmark = pytest.mark.gpu

# |logit - tau| below which the FP32 and FP64 scores may fall on either side:
# the pull features carry the FP32 precision of the residuals (~1e-3 of their
# value, see the chi2 bar), which moves a logit of unit-scale weights by ~1e-2
TIE_MLP = 2e-2


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


def _oracle_gate_scores(b, w):
    """From the FP64 oracle's best-hit finder: for every (seed, layer) where the
    candidate had two or more compatible hits, the seed and the MLP score of its
    best compatible hit by chi2."""
    r = O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
               n_best=1, dump_cap=2_000_000)
    feat, ref = r["feat"], r["feat_ref"]
    assert r["feat_count"] <= 2_000_000
    layer = np.rint(feat[:, 6] * len(b.layers)).astype(np.int64)
    key = ref[:, 0].astype(np.int64) * 1000 + layer
    order = np.lexsort((feat[:, 2], key))          # by (seed, layer), then chi2
    first = np.r_[True, key[order][1:] != key[order][:-1]]
    best = order[first & (ref[order, 2] >= 2)]
    return ref[best, 0], O.mlp_logit(w, feat[best])


def test_gate_flags_match_oracle_and_leave_tracks_unchanged():
    """Gate mode (best-hit finding with the MLP on each candidate's best
    compatible hit): the seeds it flags equal the oracle's except where a score
    is within TIE_MLP of the threshold, and the tracks are those of the same
    kernel without the gate, bit for bit."""
    from paper_1811_04141_gb300 import _native as NN
    from paper_1811_04141_gb300.api import mkf_mlp_to_bf16
    b = make_batch("dense45", [53], n_tracks=500, n_noise=60000, material=0.02, eloss=0.04)
    ctx = make_ctx(b)
    w = mlp.bf16_round(mlp.init_weights(23))
    wb = mkf_mlp_to_bf16(ctx, torch.as_tensor(w, dtype=torch.float32, device="cuda"))
    seeds, logit = _oracle_gate_scores(b, w)
    tau = float(np.quantile(logit, 0.3))  # a threshold that flags a part of the seeds
    flag_ref = np.zeros(b.n_seeds, bool)
    margin = np.full(b.n_seeds, np.inf)
    np.logical_or.at(flag_ref, seeds, logit < tau)
    np.minimum.at(margin, seeds, np.abs(logit - tau))
    from paper_1811_04141_gb300.api import feature_buffer
    gated, _ = _gpu(ctx, b, n_best=1, mlp_bf16=wb, mlp_tau=tau, mlp_mode=1)
    # the same kernel variant without the gate (feature dump, nothing pruned)
    plain, _ = _gpu(ctx, b, n_best=1, feat=feature_buffer(1 << 20))
    gated, plain = to_np(gated), to_np(plain)
    for k in ("hits", "n_hits", "counters"):
        assert np.array_equal(gated[k], plain[k]), k
    for k in ("par", "cov", "chi2"):
        assert np.array_equal(gated[k].view(np.uint32), plain[k].view(np.uint32)), k
    flag_gpu = (gated["status"] & NN.ST_AMBIG) != 0
    assert np.array_equal(gated["status"] & ~NN.ST_AMBIG, plain["status"])
    assert 0.02 < flag_ref.mean() < 0.98, flag_ref.mean()
    diff = flag_gpu != flag_ref
    assert (margin[diff] < TIE_MLP).all(), margin[diff]
    assert diff.mean() <= 2e-3


def test_seed_subset_and_seeds_where():
    """mkf_seeds_where lists exactly the seeds with the status bits, in
    ascending order; mkf_find on a seed list reproduces, for those seeds, the
    outputs of a call on every seed bit for bit and leaves the others as they
    were."""
    from paper_1811_04141_gb300 import _native as NN
    b = make_batch("dense45", [54, 55], n_tracks=700, n_noise=30000)
    ctx = make_ctx(b)
    full, d = _gpu(ctx, b, n_best=10)
    full = to_np(full)
    rng = np.random.default_rng(3)
    for n in (0, 1, 1023, 1024, 1025, 5000):
        st = torch.as_tensor(rng.integers(0, 256, n).astype(np.int32), device="cuda")
        lst, cnt = ctx.seeds_where(st, NN.ST_AMBIG | NN.ST_TRUNC)
        want = np.nonzero(st.cpu().numpy() & (NN.ST_AMBIG | NN.ST_TRUNC))[0]
        assert int(cnt.item()) == want.size and np.array_equal(lst[:want.size].cpu().numpy(), want), n
    status = np.zeros(b.n_seeds, np.int32)
    pick = rng.random(b.n_seeds) < 0.2
    status[pick] = NN.ST_AMBIG
    lst, cnt = ctx.seeds_where(torch.as_tensor(status, device="cuda"), NN.ST_AMBIG)
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    out = {k: torch.full_like(torch.as_tensor(v, device="cuda"), -7) for k, v in full.items()}
    ctx.find(bins, d["seed_hits"], d["seed_event"], n_best=10, max_out=len(b.layers) + 3, out=out, seed_list=lst,
             seed_count=cnt)
    ctx.sync()
    sub = to_np(out)
    for k, v in full.items():
        a, m = sub[k][..., pick], v[..., pick]
        assert np.array_equal(a.view(np.uint32) if a.dtype.kind == "f" else a,
                              m.view(np.uint32) if m.dtype.kind == "f" else m), k
        assert (sub[k][..., ~pick] == -7).all(), k


def test_learned_cascade_beats_plain_finder_with_material():
    """The learned cascade against the plain N-best finder on dense events with
    material (0.02 X0 and 0.04 GeV per X0 in every layer, particles scattered
    and slowed by the generator): the network is trained on the finder's own
    features with truth labels, the gate threshold is the smallest that keeps
    efficiency and fake rate within 0.5 points of the plain finder on the
    training events, and on held-out events the cascade is within 0.5 points of
    the plain finder and finds them faster (24 events)."""
    from paper_1811_04141_gb300 import learned as L
    mat = dict(material=0.02, eloss=0.04)
    tr = make_batch("dense45", list(range(2000, 2008)), truth=False, workers=8, **mat)
    ev = make_batch("dense45", list(range(12000, 12024)), truth=False, workers=8, **mat)
    ctx = make_ctx(tr)

    def prep(b):
        d = upload(b)
        d["bins"] = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
        d["hp"] = torch.as_tensor(b.hit_particle, device="cuda")
        d["sp"] = torch.as_tensor(b.seed_particle, device="cuda")
        return d

    dt, de = prep(tr), prep(ev)
    mo = len(tr.layers) + 3
    feat, ref = L.collect_features(ctx, dt["bins"], dt["seed_hits"], dt["seed_event"], 8_000_000, n_best=10,
                                   max_out=mo)
    st = L.train(ctx, feat, L.label_pairs(ref, dt["hp"], dt["sp"]), steps=1000, batch=4096, lr=2e-3)
    assert st["losses"][-1] < st["losses"][0]

    def plain(d):
        out = ctx.find(d["bins"], d["seed_hits"], d["seed_event"], n_best=10, max_out=mo)
        ctx.sync()
        return L.efficiency(out["hits"], d["hp"], d["sp"])

    def casc(d, tau):
        out, _ = L.cascade(ctx, d["bins"], d["seed_hits"], d["seed_event"], st["w_bf16"], tau, max_out=mo)
        ctx.sync()
        return L.efficiency(out["hits"], d["hp"], d["sp"])

    e0, f0 = plain(dt)
    best = L.choose_gate_tau(lambda t: casc(dt, t), e0, f0, [-6, -4, -2, -1, 0, 1, 2, 3, 4, 6])
    assert best is not None
    tau = best[0]
    ep, fp = plain(de)
    ec, fc = casc(de, tau)
    assert abs(ec - ep) <= 0.005 and fc <= fp + 0.005, (ep, ec, fp, fc)

    def ms(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        z.record()
        torch.cuda.synchronize()
        return a.elapsed_time(z) / reps

    o1 = ctx.find(de["bins"], de["seed_hits"], de["seed_event"], n_best=10, max_out=mo)
    oc, sub = L.cascade(ctx, de["bins"], de["seed_hits"], de["seed_event"], st["w_bf16"], tau, max_out=mo)
    t_plain = ms(lambda: ctx.find(de["bins"], de["seed_hits"], de["seed_event"], n_best=10, max_out=mo, out=o1))
    t_casc = ms(lambda: L.cascade(ctx, de["bins"], de["seed_hits"], de["seed_event"], st["w_bf16"], tau, max_out=mo,
                                  out=oc, subset=sub))
    print(f"cascade tau={tau}: eff {ep:.4f}->{ec:.4f} fake {fp:.5f}->{fc:.5f} ms {t_plain:.3f}->{t_casc:.3f} "
          f"flagged {int(sub[1].item()) / de['seed_hits'].shape[1]:.3f}")
    assert t_casc < t_plain


def test_cascade_replays_from_a_cuda_graph():
    """The cascade's three calls (gated best-hit finding, seed compaction,
    N-best finding of the listed seeds) need no host synchronisation: captured
    once into a CUDA graph after a first call, a replay gives the eager result."""
    from paper_1811_04141_gb300 import learned as L
    from paper_1811_04141_gb300.api import mkf_mlp_to_bf16
    b = make_batch("dense45", [57, 58], n_tracks=600, n_noise=40000, material=0.02, eloss=0.04)
    ctx = make_ctx(b)
    d = upload(b)
    mo = len(b.layers) + 3
    w = mlp.bf16_round(mlp.init_weights(29))
    wb = mkf_mlp_to_bf16(ctx, torch.as_tensor(w, dtype=torch.float32, device="cuda"))
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    eager, sub = L.cascade(ctx, bins, d["seed_hits"], d["seed_event"], wb, 0.0, max_out=mo)
    ctx.sync()
    eager = {k: v.clone() for k, v in eager.items() if v is not None}
    n_flag = int(sub[1].item())
    assert 0 < n_flag < b.n_seeds
    out = {k: torch.empty_like(v) for k, v in eager.items()}
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    with torch.cuda.stream(stream):
        L.cascade(ctx, bins, d["seed_hits"], d["seed_event"], wb, 0.0, max_out=mo, out=out, subset=sub)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        L.cascade(ctx, bins, d["seed_hits"], d["seed_event"], wb, 0.0, max_out=mo, out=out, subset=sub)
    for v in out.values():
        v.fill_(-3)
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    ctx.set_stream(torch.cuda.current_stream())
    assert int(sub[1].item()) == n_flag
    for k, v in eager.items():
        assert torch.equal(out[k].view(torch.int32), v.view(torch.int32)), k
