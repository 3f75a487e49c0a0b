"""Pins of the seed-cleaning and duplicate-track oracle (CPU only): a pure-Python
brute force over all pairs (sets, no sparse algebra), hand-worked boundary and
tie cases, and the behaviour on events with overlapping sensors (every repeated
seed removed, no other; one track kept per particle and no particle lost)."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.dedup as D
from synth import make_batch


def _brute_seeds(sh, n_hits, par, dq, de, dp):
    n = sh.shape[1]
    par = par.astype(np.float32).astype(np.float64)
    dq, de, dp = (float(np.float32(x)) for x in (dq, de, dp))
    sets = [set(int(h) for h in sh[:, i] if 0 <= h < n_hits) for i in range(n)]
    keep = []
    for i in range(n):
        k = True
        for u in range(i):
            if not (sets[i] & sets[u]):
                continue
            eta_i = -math.log(math.tan(0.5 * par[5, i]))
            eta_u = -math.log(math.tan(0.5 * par[5, u]))
            d = (par[4, i] - par[4, u] + math.pi) % (2 * math.pi) - math.pi
            if abs(par[3, i] - par[3, u]) <= dq and abs(eta_i - eta_u) <= de and abs(d) <= dp:
                k = False
        keep.append(k)
    return np.array(keep)


def _brute_tracks(hidx, n_hits, nh, c2, f):
    n = hidx.shape[1]
    c2 = c2.astype(np.float32).astype(np.float64)
    f = float(np.float32(f))
    sets = [set(int(h) for h in hidx[:, i] if 0 <= h < n_hits) for i in range(n)]
    keep = []
    for i in range(n):
        k = True
        for u in range(n):
            if u == i:
                continue
            better = nh[u] > nh[i] or (nh[u] == nh[i] and (c2[u] < c2[i] or (c2[u] == c2[i] and u < i)))
            if better and len(sets[i] & sets[u]) >= max(1.0, f * min(nh[i], nh[u])):
                k = False
        keep.append(k)
    return np.array(keep)


@pytest.mark.parametrize("seed", range(6))
def test_oracle_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, n_hits = 60, 40
    sh = rng.integers(-2, n_hits + 3, size=(3, n))
    par = np.zeros((6, n))
    par[3] = rng.choice([-1.0, 1.0], n) * rng.uniform(0.2, 0.4, n)
    par[4] = rng.uniform(-math.pi, math.pi, n)
    par[5] = rng.uniform(0.3, 2.8, n)
    for tol in ((0.15, 0.02, 0.02), (1.0, 5.0, 7.0), (0.0, 0.0, 0.0)):
        assert (D.clean_seeds(sh, n_hits, par, *tol) == _brute_seeds(sh, n_hits, par, *tol)).all()
    hidx = rng.integers(-1, n_hits, size=(8, n))
    nh = rng.integers(3, 9, n)
    c2 = rng.integers(0, 4, n).astype(np.float64)  # many exact chi2 ties
    for f in (0.0, 0.3, 0.5, 1.0):
        assert (D.dedup_tracks(hidx, n_hits, nh, c2, f) == _brute_tracks(hidx, n_hits, nh, c2, f)).all()


def test_hand_cases():
    # seeds (columns) 0 and 1 share hit 7; seed 2 shares hit 9 with seed 1 only
    sh = np.array([[7, 7, 20], [3, 9, 9], [4, 5, 6]])
    par = np.zeros((6, 3))
    par[5] = 1.0
    par[3] = [0.5, 0.625, 0.75]              # |d q/pT| 0.125 (0-1), 0.125 (1-2), 0.25 (0-2), exact in float
    # exactly at the tolerance counts as a duplicate (<=); seed 2 has a duplicate
    # (seed 1, a lower index) and is dropped even though seed 1 is dropped too
    keep = D.clean_seeds(sh, 30, par, max_dqpt=0.125, max_deta=0.02, max_dphi=0.02)
    assert keep.tolist() == [True, False, False]
    keep = D.clean_seeds(sh, 30, par, max_dqpt=0.1, max_deta=0.02, max_dphi=0.02)
    assert keep.tolist() == [True, True, True]
    # phi wraps: 3.14 and -3.14 differ by 0.0032
    par[3] = 0.5
    par[4] = [3.14, -3.14, 0.0]
    keep = D.clean_seeds(sh, 30, par, max_dqpt=0.1, max_deta=0.02, max_dphi=0.01)
    assert keep.tolist() == [True, False, True]
    # tracks: 0 (5 hits) and 1 (4 hits) share 2 = 0.5 x 4 -> 1 dropped; 2 shares 1 hit with 0
    hidx = np.array([[1, 2, 3, 4, 5], [4, 5, 11, 12, -1], [5, 20, 21, 22, 23]]).T.copy()
    nh = np.array([5, 4, 5])
    c2 = np.array([3.0, 1.0, 2.0])
    assert D.dedup_tracks(hidx, 30, nh, c2, 0.5).tolist() == [True, False, True]
    # with min_frac 0.125 a single shared hit is enough (need = max(1, 0.125 x 5)):
    # track 0 then loses to track 2 (as many hits, lower chi2).  (0.2 would not
    # do: float32(0.2) x 5 is just above 1.)
    assert D.dedup_tracks(hidx, 30, nh, c2, 0.125).tolist() == [False, False, True]
    assert D.dedup_tracks(hidx, 30, nh, c2, 0.2).tolist() == [True, False, True]
    # exact chi2 tie: the lower index wins
    c2 = np.array([2.0, 1.0, 2.0])
    assert D.dedup_tracks(hidx, 30, nh, c2, 0.125).tolist() == [True, False, False]


def _seed_fit(b):
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz.astype(np.float64), b.layer, b.seed_hits)
    return r["par"].astype(np.float32), r["status"]


@pytest.mark.parametrize("cfg", ["find20", "dense45"])
def test_seed_cleaning_on_overlap_events(cfg):
    """Every repeated seed of a particle (one hit replaced by its twin) is removed;
    seeds of different particles never are (default tolerances; on dense45 the
    inner disks' short lever arm spreads the 3-hit q/pT of a repeated seed up to
    0.2 c/GeV from its original)."""
    b = make_batch(cfg, [0, 1], n_tracks=400, overlap=0.15)
    par, st = _seed_fit(b)
    assert (st == 0).all()
    keep = D.clean_seeds(b.seed_hits, b.n_hits, par)
    dup = b.seed_dup_of >= 0
    assert dup.sum() > 50
    assert not keep[dup].any()
    assert keep[~dup].all()


def test_track_dedup_after_finding_with_repeated_seeds():
    """Finding from every seed (repeated ones included) gives several tracks per
    particle; removal keeps one per particle and loses none."""
    b = make_batch("find20", [2], n_tracks=300, overlap=0.15)
    geo = O.geometry_for(b)
    r = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=10,
               max_out=len(b.layers) + 3)
    keep = D.dedup_tracks(r["hits"], b.n_hits, r["n_hits"], r["chi2"], 0.5)
    hits = r["hits"]
    owner = np.where(hits >= 0, b.hit_particle[np.maximum(hits, 0)], -2)
    frac = (owner == b.seed_particle[None, :]).sum(0) / np.maximum((hits >= 0).sum(0), 1)
    matched = frac >= 0.75
    found_before = set(b.seed_particle[matched])
    found_after = set(b.seed_particle[matched & keep])
    assert found_after == found_before
    per_particle = np.bincount(b.seed_particle[matched & keep], minlength=b.particle_nhits.size)
    assert per_particle.max() == 1
    assert (~keep).sum() >= (b.seed_dup_of >= 0).sum() * 0.9
