"""Pins of the oracle's r-z material map (Sec. 2.1: radiation and interaction
lengths from two-dimensional arrays indexed in r and z): the cell that holds a
crossing point, checked by brute force over the cell edges; a uniform map
equal to the same material given per layer; and the pulls of the fit on tracks
that the generator scatters and slows with the map's own values at each
crossing."""
import bisect

import numpy as np

import oracle as O
from synth import make_batch
from tests.test_oracle_pins import _last_hits, _pulls

R_MAX, Z_MIN, Z_MAX = 110.0, -130.0, 130.0


def _map(nr=7, nz=9, x0=None, eloss=None):
    return dict(r_max=R_MAX, z_min=Z_MIN, z_max=Z_MAX, x0=np.full((nr, nz), 0.03) if x0 is None else x0,
                eloss=eloss)


def _cell(edges, v):
    """Index of the cell of sorted edges [e0, ..., en] holding v; outside: the edge cell."""
    i = bisect.bisect_right(list(edges), v) - 1
    return min(max(i, 0), len(edges) - 2)


def test_map_lookup_cell_by_brute_force():
    """Each cell's x0 encodes its index; the noise the oracle adds at a point
    equals the noise of that x0 given to the layer directly, for the cell found
    by bisection over the edges (points outside the map included)."""
    nr, nz = 6, 11
    x0 = 1e-3 * (1.0 + np.arange(nr * nz, dtype=np.float64).reshape(nr, nz))
    b = make_batch("fit10", [0], n_tracks=1)
    geo = O.Geometry(b.layers, b.bz, material_map=_map(nr, nz, x0))
    r_edges = np.linspace(0.0, R_MAX, nr + 1)
    z_edges = np.linspace(Z_MIN, Z_MAX, nz + 1)
    rng = np.random.default_rng(3)
    for _ in range(60):
        l = int(rng.integers(0, len(b.layers)))
        R = b.layers[l]["r_or_z"]
        z = rng.uniform(-160.0, 160.0)
        ph = rng.uniform(-np.pi, np.pi)
        p = np.array([R * np.cos(ph), R * np.sin(ph), z, 0.7, ph + 0.1, 1.1])
        want = x0[_cell(r_edges, R), _cell(z_edges, z)]
        layers = [dict(d, x0=(want if i == l else 0.0)) for i, d in enumerate(b.layers)]
        ref = O.scattering(O.Geometry(layers, b.bz), l, p)
        assert np.array_equal(O.scattering(geo, l, p), ref), (l, R, z)


def test_uniform_map_equals_material_per_layer():
    b = make_batch("fit10", [16], n_tracks=300, material=0.03, eloss=0.15)
    per_layer = O.geometry_for(b)
    bare = [{k: v for k, v in d.items() if k not in ("x0", "eloss")} for d in b.layers]
    mapped = O.Geometry(bare, b.bz, material_map=_map(eloss=np.full((7, 9), 0.15)))
    a = O.fit(per_layer, b.xyz64, b.layer, b.track_hits)
    m = O.fit(mapped, b.xyz64, b.layer, b.track_hits)
    for k in ("par", "cov", "chi2", "ndf", "status"):
        assert np.array_equal(a[k], m[k]), k


def _graded_map():
    """Thin in the centre, three times thicker towards |z| = 130 and twice as
    thick in the outer radii; energy loss (0.04 GeV per radiation length, about
    silicon's) in the outer half only."""
    nr, nz = 7, 9
    zc = np.linspace(Z_MIN, Z_MAX, nz + 1)
    zc = 0.5 * (zc[1:] + zc[:-1])
    rc = np.linspace(0.0, R_MAX, nr + 1)
    rc = 0.5 * (rc[1:] + rc[:-1])
    x0 = 0.01 * (1.0 + 2.0 * (np.abs(zc)[None, :] / Z_MAX)) * (1.0 + (rc[:, None] > 50.0))
    el = np.where(rc[:, None] > 50.0, 0.04, 0.0) * np.ones((1, nz))
    return _map(nr, nz, x0, el)


def test_fit_with_graded_map_pulls_and_chi2():
    """Tracks scattered and slowed with a graded map: with that map the pulls
    are N(0, 1) and chi2/ndf = 1; with the map's mean thickness in every layer
    instead, chi2/ndf moves away from 1."""
    mm = _graded_map()
    b = make_batch("fit10", list(range(6)), n_tracks=1000, material_map=mm)
    geo = O.geometry_for(b)
    assert geo.material_map is mm
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    ok = r["status"] == 0
    truth = b.true_state[:, _last_hits(b)][:, ok]
    for i, pull in _pulls(r["par"][:, ok], truth, r["cov"][:, ok]).items():
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i
    assert abs(r["chi2"][ok].sum() / r["ndf"][ok].sum() - 1) < 0.03
    flat = [dict(d, x0=float(mm["x0"].mean()), eloss=float(mm["eloss"].mean())) for d in b.layers]
    r0 = O.fit(O.Geometry(flat, b.bz), b.xyz64, b.layer, b.track_hits)
    assert abs(r0["chi2"][ok].sum() / r0["ndf"][ok].sum() - 1) > 0.05


def test_eloss_covariance_is_the_derivative_of_the_loss_map():
    """The covariance transform of the energy loss against the derivative of
    the loss map itself (central differences of the state it returns), for loss
    and gain, slow and fast, central and forward tracks: d(q/pT')/d(q/pT) to
    1e-6 (the path through the layer does not depend on q/pT), and the whole
    transform J C J^T to 2e-2, the differences in theta also moving the path
    x0 / |cos a| that the transform holds fixed."""
    b = make_batch("fit10", [0], n_tracks=1)
    layers = [dict(d, x0=0.05, eloss=0.2) for d in b.layers]
    geo = O.Geometry(layers, b.bz)
    rng = np.random.default_rng(11)
    A = rng.standard_normal((6, 6))
    Cm = A @ A.T + 6 * np.eye(6)
    e3 = np.zeros((6, 6))
    e3[3, 3] = 1.0
    R = layers[4]["r_or_z"]
    for w, th, sign in ((2.0, 1.2, 1.0), (-1.5, 0.6, 1.0), (0.3, 1.5, 1.0), (1.8, 2.3, -1.0), (-0.9, 1.0, -1.0)):
        p = np.array([R * np.cos(0.3), R * np.sin(0.3), 12.0, w, 0.35, th])
        q, C2 = O.eloss(geo, 4, p, Cm, sign)
        assert abs(q[3] / w - 1) > 1e-3  # the loss does act here
        J = np.eye(6)
        for j, e in ((3, 1e-6 * abs(w)), (5, 1e-6)):
            a, bb = p.copy(), p.copy()
            a[j] += e
            bb[j] -= e
            J[:, j] = (O.eloss(geo, 4, a, Cm, sign)[0] - O.eloss(geo, 4, bb, Cm, sign)[0]) / (2 * e)
        a33 = np.sqrt(O.eloss(geo, 4, p, e3, sign)[1][3, 3])
        assert abs(a33 - abs(J[3, 3])) < 1e-6 * abs(J[3, 3]), (w, th, sign, a33, J[3, 3])
        want = J @ Cm @ J.T
        assert np.abs(C2 - want).max() < 2e-2 * np.abs(want).max(), (w, th, sign, C2 - want)
