"""Pins of the oracle's learned-pruning path (or_find with MLP weights): the
scoring function equals the separately pinned MLP oracle (oracle/mlp.py), the 12
features the finder computes for a (candidate, compatible hit) pair equal the
values rebuilt from the exported single-step calls (seed, propagate, transport,
update) and the feature definitions, and pruning that drops nothing reproduces
the plain finder exactly.  A planted mistake in the features (two columns
swapped, a wrong ndf) fails the feature check."""
import numpy as np

import oracle as O
from oracle import mlp
from synth import make_batch

CUT = 30.0


def test_finder_score_equals_mlp_oracle():
    rng = np.random.default_rng(5)
    for _ in range(3):
        w = mlp.bf16_round(mlp.init_weights(int(rng.integers(1 << 30))) * rng.uniform(0.5, 3.0))
        X = rng.normal(size=(500, 12)) * rng.uniform(0.1, 5.0, size=12)
        a = O.mlp_logit(w, X)
        b = mlp.forward(w, X)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(b).max())
    # all hidden units off: the output bias alone
    w = np.zeros(mlp.N_PARAMS)
    w[-1] = 0.75
    w[768:832] = -1.0
    assert np.all(O.mlp_logit(w, rng.normal(size=(4, 12))) == 0.75)


def _rebuild_features(geo, b, hits_found, seed_index, hit, n_layers):
    """Features of the pair (candidate of seed `seed_index`, `hit`) from the
    seed state, the Kalman fit through the seed hits and the hits the best-hit
    finder chose on earlier layers, and the prediction at the hit's layer."""
    X = b.xyz.astype(np.float64)
    found = [h for h in hits_found[:, seed_index] if h >= 0]
    layer = int(b.layer[hit])
    j = next(k for k, h in enumerate(found) if b.layer[h] == layer)
    s = O.seed(geo, X[:, found[0]], X[:, found[1]], X[:, found[2]], b.layer[found[0]])
    p, Cm = s
    chi2 = 0.0
    for k in range(j):
        h = found[k]
        if k > 0:
            q, J, _ = O.propagate(geo, p, b.layer[h])
            Cm = O.transport(J, Cm)
            p = q
        p, Cm, c2, *_ = O.update(geo, b.layer[h], X[:, h], p, Cm)
        chi2 += c2
    q, J, _ = O.propagate(geo, p, layer)
    Cp = O.transport(J, Cm)
    _, _, x2, r, S, _ = O.update(geo, layer, X[:, hit], q, Cp)
    n = j
    su, sv = np.sqrt(S[0, 0]), np.sqrt(S[1, 1])
    return np.array([r[0] / su, r[1] / sv, x2 / CUT, chi2 / max(1, 2 * n - 5), 0.1 * n, 0.0, layer / n_layers,
                     float(b.layers[layer]["kind"] == 1), q[3], np.arcsinh(np.cos(q[5]) / np.sin(q[5])) / 3.0,
                     np.log10(su), np.log10(sv)])


def _feature_mismatch(feat, rebuilt):
    """Largest |difference| / (1e-9 |value| + 1e-12) per feature column."""
    return (np.abs(feat - rebuilt) / (1e-9 * np.abs(rebuilt) + 1e-12)).max(axis=0)


def test_features_equal_single_step_rebuild():
    # clean events (no noise, no inefficiency): with N = 1 each seed's candidate
    # follows the hits it found, so its state at any layer is the fit through them
    b = make_batch("find20", [61, 62], n_tracks=150, n_noise=0, ineff=0.0)
    geo = O.geometry_as_loaded(b)
    r = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=1,
               chi2_cut=CUT, dump_cap=200000)
    feat, ref = r["feat"], r["feat_ref"]
    assert feat.shape[0] > 1000
    # rows of candidates without a miss (feature 5 = 0), on both kinds of layer
    rng = np.random.default_rng(0)
    rows = rng.choice(np.nonzero(feat[:, 5] == 0.0)[0], 150, replace=False)
    rebuilt = np.array([_rebuild_features(geo, b, r["hits"], int(ref[i, 0]), int(ref[i, 1]), geo.n) for i in rows])
    assert set(rebuilt[:, 7]) == {0.0, 1.0}
    assert (_feature_mismatch(feat[rows], rebuilt) <= 1.0).all(), _feature_mismatch(feat[rows], rebuilt)
    # planted mistakes are caught: two columns swapped, ndf of feature 3 off by one
    swapped = feat[rows].copy()
    swapped[:, [0, 1]] = swapped[:, [1, 0]]
    assert _feature_mismatch(swapped, rebuilt)[:2].max() > 1.0
    bad_ndf = rebuilt.copy()
    n = rebuilt[:, 4] * 10
    bad_ndf[:, 3] = rebuilt[:, 3] * np.maximum(1, 2 * n - 5) / np.maximum(1, 2 * n - 4)
    assert _feature_mismatch(feat[rows], bad_ndf)[3] > 1.0


def test_pruning_that_drops_nothing_is_the_plain_finder():
    b = make_batch("dense45", [63], n_tracks=300, n_noise=40000)
    geo = O.geometry_as_loaded(b)
    x = b.xyz.astype(np.float64)
    w = mlp.bf16_round(mlp.init_weights(7))
    plain = O.find(geo, x, b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=10)
    pruned = O.find(geo, x, b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=10, mlp_w=w,
                    mlp_tau=-np.inf)
    for k in ("hits", "n_hits", "status", "counters"):
        assert np.array_equal(plain[k], pruned[k]), k
    for k in ("par", "cov", "chi2"):
        assert np.array_equal(plain[k], pruned[k], equal_nan=True), k
    # and a threshold above every score drops every hit of a candidate with two or
    # more compatible hits: fewer Kalman updates than the plain finder
    cut_all = O.find(geo, x, b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=10, mlp_w=w,
                     mlp_tau=np.inf)
    assert cut_all["counters"][2].sum() < plain["counters"][2].sum()
