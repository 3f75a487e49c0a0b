"""Oracle for seed cleaning and duplicate-track removal (TEST INFRASTRUCTURE
ONLY: only the tests, the smoke check and the bench's CPU baseline may use it).

Sec. 2.2 describes seed cleaning as removing repeated seeds of one particle
using the identity of their hits and their fitted pT, eta and phi; Sec. 3
names the removal of duplicate tracks (several seeds per particle) as missing
post-processing.  The paper fixes no rule; the readings written out here are:

  seeds   two seeds are duplicates when they share at least one hit and their
          fitted parameters agree: |d(q/pT)| <= max_dqpt, |d eta| <= max_deta,
          |d phi| (wrapped) <= max_dphi; a seed is dropped when a duplicate with
          a lower index exists;
  tracks  two tracks are duplicates when the hits they share number at least
          min_frac x (hits of the shorter one) (and at least one); a track is
          dropped when a duplicate that is better exists: more hits, then lower
          chi2, then lower index.

Each decision looks only at the other item, never at whether that item is
itself dropped, so the result does not depend on any processing order.  The
shared-hit counts of all pairs are one sparse product of the item x hit
incidence matrix with its transpose; everything else is a direct comparison,
done in double on the given (float32) inputs and on the float32 values of the
tolerances (the values a float argument carries).
"""
import numpy as np
import scipy.sparse as sp


def _incidence(hit_lists, n_hits):
    """hit_lists [k][n] (-1 = none) -> CSR items x hits (0/1, duplicates in a list counted once)."""
    k, n = hit_lists.shape
    items = np.broadcast_to(np.arange(n), (k, n)).ravel()
    hits = hit_lists.ravel()
    ok = (hits >= 0) & (hits < n_hits)
    m = sp.csr_matrix((np.ones(int(ok.sum()), dtype=np.int64), (items[ok], hits[ok])), shape=(n, n_hits))
    m.sum_duplicates()
    m.data[:] = 1  # a hit listed twice by one item counts once
    return m


def _shared_pairs(hit_lists, n_hits):
    """(i, u, shared) for every ordered pair i != u of items sharing >= 1 hit."""
    a = _incidence(np.asarray(hit_lists), int(n_hits))
    s = (a @ a.T).tocoo()
    off = s.row != s.col
    return s.row[off], s.col[off], s.data[off]


def clean_seeds(seed_hits, n_hits, seed_par, max_dqpt=0.5, max_deta=0.02, max_dphi=0.02):
    """keep [n] (bool) for seeds seed_hits [3][n] with fitted states seed_par [6][n]
    (q/pT, phi, theta in rows 3, 4, 5)."""
    seed_hits = np.asarray(seed_hits)
    n = seed_hits.shape[1]
    par = np.asarray(seed_par, dtype=np.float32).astype(np.float64)
    max_dqpt, max_deta, max_dphi = (float(np.float32(x)) for x in (max_dqpt, max_deta, max_dphi))
    i, u, _ = _shared_pairs(seed_hits, n_hits)
    eta = -np.log(np.tan(0.5 * par[5]))
    dphi = np.abs(np.remainder(par[4, i] - par[4, u] + np.pi, 2 * np.pi) - np.pi)
    dup = (np.abs(par[3, i] - par[3, u]) <= max_dqpt) & (np.abs(eta[i] - eta[u]) <= max_deta) & (dphi <= max_dphi)
    keep = np.ones(n, dtype=bool)
    keep[i[dup & (u < i)]] = False
    return keep


def dedup_tracks(hit_idx, n_hits, track_nhits, chi2, min_frac=0.5):
    """keep [n] (bool) for tracks hit_idx [max_out][n] (-1 = none) with hit counts
    track_nhits [n] and chi2 [n]."""
    hit_idx = np.asarray(hit_idx)
    n = hit_idx.shape[1]
    nh = np.asarray(track_nhits).astype(np.int64)
    c2 = np.asarray(chi2, dtype=np.float32).astype(np.float64)
    min_frac = float(np.float32(min_frac))
    i, u, shared = _shared_pairs(hit_idx, n_hits)
    need = np.maximum(1.0, min_frac * np.minimum(nh[i], nh[u]))
    dup = shared >= need
    better = (nh[u] > nh[i]) | ((nh[u] == nh[i]) & ((c2[u] < c2[i]) | ((c2[u] == c2[i]) & (u < i))))
    keep = np.ones(n, dtype=bool)
    keep[i[dup & better]] = False
    return keep
