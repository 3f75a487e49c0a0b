"""Pins of the oracle's smoother (the state at every hit from all of a track's
hits: the forward filter's state after each hit combined with the backward
filter's prediction there).  Against what the oracle's smoother does not
compute itself: the generator's true state at each hit (noise-free hits give
it back; smeared hits give pulls N(0, 1) at every hit, with and without
material), the forward fit at the last hit, and, without material, the final
fitted state moved back along the helix to each hit."""
import numpy as np
import pytest

import oracle as O
from synth import make_batch
from tests.test_oracle_pins import _pulls, wrap


def _hit_truth(b):
    """[max_hits, 6, n] true states per row of track_hits (NaN where none)."""
    th = b.track_hits
    out = np.full((th.shape[0], 6, th.shape[1]), np.nan)
    m = th >= 0
    for k in range(th.shape[0]):
        out[k][:, m[k]] = b.true_state[:, th[k][m[k]]]
    return out


def test_smooth_noise_free_recovers_truth():
    for cfg in ("fit10", "find20"):
        b = make_batch(cfg, [4], n_tracks=200, smear=False)
        geo = O.geometry_for(b)
        r = O.fit_smooth(geo, b.xyz64, b.layer, b.track_hits)
        ok = r["status"] == 0
        truth = _hit_truth(b)
        m = (b.track_hits >= 0) & ok[None, :]
        d = r["par"] - truth
        d[:, 4] = wrap(d[:, 4])
        for i, tol in enumerate((1e-6, 1e-6, 1e-6, 1e-6, 1e-7, 1e-7)):
            assert np.abs(d[:, i][m]).max() < tol * max(1.0, np.abs(truth[:, i][m]).max()), (cfg, i)


def test_smooth_last_hit_is_the_forward_fit():
    b = make_batch("find20", [5], n_tracks=300)
    geo = O.geometry_for(b)
    r = O.fit_smooth(geo, b.xyz64, b.layer, b.track_hits)
    f = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    assert np.array_equal(r["chi2"], f["chi2"]) and np.array_equal(r["ndf"], f["ndf"])
    ok = (r["status"] == 0) & (f["status"] == 0)
    last = np.array([np.nonzero(b.track_hits[:, t] >= 0)[0][-1] for t in range(b.n_seeds)])
    t = np.nonzero(ok)[0]
    assert np.array_equal(r["par"][last[t], :, t].T, f["par"][:, t])
    assert np.array_equal(r["cov"][last[t], :, t].T, f["cov"][:, t])


@pytest.mark.parametrize("material", [0.0, 0.03])
def test_smooth_pulls_at_every_hit(material):
    """Pulls of the smoothed state against the true state at every hit are
    N(0, 1) (z, q/pT, phi, theta), pooled over the hits of 6000 tracks; the
    smoothed errors are far below the forward filter's at the first hits."""
    b = make_batch("fit10", list(range(6)), n_tracks=1000, material=material, eloss=0.0)
    geo = O.geometry_for(b)
    r = O.fit_smooth(geo, b.xyz64, b.layer, b.track_hits)
    ok = r["status"] == 0
    truth = _hit_truth(b)
    m = (b.track_hits >= 0) & ok[None, :]
    par = np.transpose(r["par"], (1, 0, 2))[:, m]
    cov = np.transpose(r["cov"], (1, 0, 2))[:, m]
    tru = np.transpose(truth, (1, 0, 2))[:, m]
    for i, pull in _pulls(par, tru, cov).items():
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i
    # at the third hit the smoothed q/pT is known about as well as at the last
    k3 = np.array([np.nonzero(b.track_hits[:, t] >= 0)[0][2] for t in range(b.n_seeds)])
    t = np.nonzero(ok)[0]
    f3 = O.fit(geo, b.xyz64, b.layer, np.where(np.arange(b.track_hits.shape[0])[:, None] <= k3[None, :],
                                                 b.track_hits, -1))
    assert np.median(r["cov"][k3[t], 9, t] / f3["cov"][9, t]) < 0.1


def test_smooth_without_material_is_the_fit_moved_back():
    """Without material the state is a deterministic function of its value at
    any surface: the smoothed state at each hit equals the final fitted state
    moved back along the helix to that hit's layer, to a small fraction of its
    standard deviation."""
    b = make_batch("fit10", [7], n_tracks=300)
    geo = O.geometry_for(b)
    r = O.fit_smooth(geo, b.xyz64, b.layer, b.track_hits)
    f = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    ok = np.nonzero((r["status"] == 0) & (f["status"] == 0))[0]
    worst = 0.0
    for t in ok[:100]:
        rows = np.nonzero(b.track_hits[:, t] >= 0)[0]
        q = f["par"][:, t].copy()
        q[3], q[4], q[5] = -q[3], wrap(q[4] + np.pi), np.pi - q[5]  # turned around
        for k in rows[::-1][1:]:
            mv = O.propagate(geo, q, b.layer[b.track_hits[k, t]])
            assert mv is not None
            q = mv[0]
            back = q.copy()
            back[3], back[4], back[5] = -back[3], wrap(back[4] + np.pi), np.pi - back[5]
            sig = np.sqrt(np.diag(O.unpack21(r["cov"][k][:, t:t + 1])[0]))
            d = r["par"][k, :, t] - back
            d[4] = wrap(d[4])
            worst = max(worst, np.max(np.abs(d[2:]) / sig[2:]))
    assert worst < 0.05
