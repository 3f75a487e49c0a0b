"""Pins of the oracle's propagation in the parameterised field (Sec. 2.1: a
constant or a parameterised field, chosen per propagation): fourth-order
Runge-Kutta steps along the path, Newton steps onto the surface and the
Jacobian of that map by central differences.

They pin it to what does not come from the oracle: Maxwell's equations for
the field, the closed-form helix in a uniform field, scipy's eighth-order
Dormand-Prince integrator with event location for the trajectory and (by its
own finite differences) for the Jacobian, and the pulls of the fit on tracks
the generator moves through the field with its own integrator."""
import numpy as np
import pytest

import oracle as O
from synth import K_FIELD, make_batch
from synth.events import solenoid_field
from tests.test_oracle_pins import _first_hits, _last_hits, _pulls, wrap

ALPHA = 1e-5  # 1/cm^2: Bz 10 % lower at z = +-100 cm, 5 % higher at r = 100 cm

# Truncation of the oracle's Runge-Kutta steps (at most 0.05 rad of turning
# each): the global error of a fourth-order method is about n (a^5 / 120) rho
# for n steps of angle a on a circle of radius rho, 3e-6 cm for a 0.6 GeV track
# taking 12 steps to the disk, and up to 2e-7 rad in direction for the
# slowest tracks (0.5 GeV) over a layer gap: positions to 1e-5 cm (0.5 % of a
# 20 um resolution), angles and relative q/pT to 5e-7.
TOL_POS, TOL_ANG = 1e-5, 5e-7

scipy_integrate = pytest.importorskip("scipy.integrate")


def _layers_cyl_disk():
    return [dict(kind=0, r_or_z=30.0, lo=-150.0, hi=150.0, sigma_u=2e-3, sigma_v=1e-2),
            dict(kind=0, r_or_z=45.0, lo=-150.0, hi=150.0, sigma_u=2e-3, sigma_v=1e-2),
            dict(kind=1, r_or_z=120.0, lo=5.0, hi=110.0, sigma_u=2e-3, sigma_v=1e-2)]


def _scipy_move(bz, alpha, p, kind, rz):
    """The state p moved onto the surface (r = rz or z = rz) by DOP853 with a
    terminal event, tolerances near double precision."""
    st = np.sin(p[5])
    y0 = np.array([p[0], p[1], p[2], st * np.cos(p[4]), st * np.sin(p[4]), np.cos(p[5])])
    lam = p[3] * st

    def rhs(_s, y):
        bx, by, bzz = solenoid_field(bz, alpha, y[0], y[1], y[2])
        k = K_FIELD * lam
        return [y[3], y[4], y[5], k * (y[4] * bzz - y[5] * by), k * (y[5] * bx - y[3] * bzz),
                k * (y[3] * by - y[4] * bx)]

    def ev(_s, y):
        return (np.hypot(y[0], y[1]) - rz) if kind == 0 else (y[2] - rz)

    ev.terminal = True
    sol = scipy_integrate.solve_ivp(rhs, (0.0, 1000.0), y0, method="DOP853", events=ev, rtol=1e-13, atol=1e-13)
    y = sol.y_events[0][0]
    tt = np.hypot(y[3], y[4]) / np.linalg.norm(y[3:6])
    return np.array([y[0], y[1], y[2], lam / tt, np.arctan2(y[4], y[3]), np.arctan2(tt, y[5] / np.linalg.norm(y[3:6]))])


def _inside(layer, q):
    """The crossing lies within the layer's extent (where a hit can be)."""
    c = q[2] if layer["kind"] == 0 else np.hypot(q[0], q[1])
    return layer["lo"] <= c <= layer["hi"]


def _states():
    """States on the first cylinder (r = 30) heading out: pT 0.6-20 GeV, both
    charges, polar angles from 40 to 140 degrees."""
    rng = np.random.default_rng(5)
    out = []
    for k in range(24):
        ph = rng.uniform(-np.pi, np.pi)
        th = rng.uniform(0.7, 2.4)
        w = rng.choice([-1, 1]) / rng.uniform(0.6, 20.0)
        out.append(np.array([30 * np.cos(ph), 30 * np.sin(ph), rng.uniform(-40, 40), w,
                             wrap(ph + rng.uniform(-0.2, 0.2)), th]))
    return out


def test_field_is_divergence_and_curl_free():
    geo = O.Geometry(_layers_cyl_disk(), 3.8, field_alpha=ALPHA)
    assert np.allclose(O.field(geo, [0, 0, 0]), [0, 0, 3.8], atol=0)
    e = 1e-3
    for r in ([10.0, -20.0, 50.0], [-70.0, 30.0, -110.0]):
        D = np.zeros((3, 3))  # D[i, j] = dB_i / dx_j
        for j in range(3):
            a, b = np.array(r, float), np.array(r, float)
            a[j] += e
            b[j] -= e
            D[:, j] = (O.field(geo, a) - O.field(geo, b)) / (2 * e)
        scale = np.abs(D).max()
        assert abs(np.trace(D)) < 1e-9 * scale
        curl = [D[2, 1] - D[1, 2], D[0, 2] - D[2, 0], D[1, 0] - D[0, 1]]
        assert np.abs(curl).max() < 1e-9 * scale
        assert np.allclose(O.field(geo, r), solenoid_field(3.8, ALPHA, *r), rtol=1e-14)


def test_rk_in_uniform_field_is_the_helix():
    """alpha = 0 integrated numerically vs the closed-form helix and its
    analytic Jacobian (the uniform-field mode of the same geometry)."""
    L = _layers_cyl_disk()
    helix = O.Geometry(L, 3.8)
    rk = O.Geometry(L, 3.8, field_alpha=0.0)
    n = 0
    for p in _states():
        for l in (1, 2):
            a, b = O.propagate(helix, p, l), O.propagate(rk, p, l)
            assert (a is None) == (b is None)
            if a is None or not _inside(L[l], a[0]):
                continue
            n += 1
            d = a[0] - b[0]
            d[4] = wrap(d[4])
            assert np.abs(d[:3]).max() < TOL_POS, (p, l, d)
            assert abs(d[3]) < TOL_ANG * abs(p[3]) and np.abs(d[4:]).max() < TOL_ANG, (p, l, d)
            Ja, Jb = a[1], b[1]
            assert np.abs(Ja - Jb).max() < 2e-6 * np.abs(Ja).max(), (p, l, Ja - Jb)
    assert n >= 16


def test_rk_against_dop853_with_events():
    """The oracle's steps (a few per layer gap) land within their truncation
    error of DOP853 at 1e-13 tolerance, on cylinders and on a disk."""
    geo = O.Geometry(_layers_cyl_disk(), 3.8, field_alpha=ALPHA)
    n = 0
    for p in _states():
        for l in (1, 2):
            r = O.propagate(geo, p, l)
            if r is None or not _inside(geo.layers[l], r[0]):
                continue
            n += 1
            ref = _scipy_move(3.8, ALPHA, p, geo.kind[l], geo.rz[l])
            d = r[0] - ref
            d[4] = wrap(d[4])
            assert np.abs(d[:3]).max() < TOL_POS, (p, l, d)
            assert abs(d[3]) < TOL_ANG * abs(p[3]) and np.abs(d[4:]).max() < TOL_ANG, (p, l, d)
    assert n >= 16


def test_rk_jacobian_against_dop853_differences():
    """The Jacobian of the oracle's map vs central differences of DOP853's (its
    own steps, 1e-13 tolerance): the surface constraint, the parameter
    conversions and the field's bending of theta and q/pT all enter both."""
    geo = O.Geometry(_layers_cyl_disk(), 3.8, field_alpha=ALPHA)
    eps = np.array([1e-3, 1e-3, 1e-3, 0.0, 1e-5, 1e-5])
    for p in _states()[:5]:
        for l in (1, 2):
            r = O.propagate(geo, p, l)
            if r is None or not _inside(geo.layers[l], r[0]):
                continue
            J = r[1]
            e = eps.copy()
            e[3] = 1e-5 * abs(p[3])
            for j in range(6):
                a, b = p.copy(), p.copy()
                a[j] += e[j]
                b[j] -= e[j]
                d = _scipy_move(3.8, ALPHA, a, geo.kind[l], geo.rz[l]) - _scipy_move(3.8, ALPHA, b, geo.kind[l],
                                                                                      geo.rz[l])
                d[4] = wrap(d[4])
                col = d / (2 * e[j])
                tol = 1e-5 * max(1.0, np.abs(col).max())
                assert np.abs(col - J[:, j]).max() < tol, (p, l, j, col, J[:, j])


def test_generator_crossings_against_dop853():
    """The generator's own integrator (fixed 0.5 cm steps) vs DOP853 from the
    vertex: crossing points within 1e-6 cm."""
    b = make_batch("fit10", [3], n_tracks=20, field_alpha=ALPHA, smear=False)
    for t in range(5):
        hh = b.track_hits[:, t]
        hh = hh[hh >= 0]
        p0 = b.particle_par[:, b.seed_particle[t]]
        for h in hh[:4]:
            l = b.layer[h]
            ref = _scipy_move(b.bz, ALPHA, p0, 0, b.layers[l]["r_or_z"])
            assert np.abs(ref[:3] - b.true_xyz[:, h]).max() < 1e-6
            assert abs(ref[3] - b.true_state[3, h]) < 1e-8 * abs(ref[3])
            p0 = ref


def test_fit_in_parameterised_field_pulls_and_chi2():
    """Tracks moved through the field by the generator: with the parameterised
    field the filter's pulls are N(0, 1) and chi2/ndf = 1; with the uniform
    field the same hits give chi2/ndf far above 1."""
    b = make_batch("fit10", list(range(4)), n_tracks=1000, field_alpha=ALPHA)
    geo = O.geometry_for(b)
    assert geo.field_kind == 1 and geo.alpha == ALPHA
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    ok = r["status"] == 0
    assert ok.mean() > 0.99
    truth = b.true_state[:, _last_hits(b)][:, ok]
    for i, pull in _pulls(r["par"][:, ok], truth, r["cov"][:, ok]).items():
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i
    assert abs(r["chi2"][ok].sum() / r["ndf"][ok].sum() - 1) < 0.03
    r0 = O.fit(O.Geometry(b.layers, b.bz), b.xyz64, b.layer, b.track_hits)
    assert r0["chi2"][ok].sum() / r0["ndf"][ok].sum() > 10


def test_backfit_in_parameterised_field_pulls():
    b = make_batch("fit10", list(range(4)), n_tracks=1000, field_alpha=ALPHA)
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    rb = O.fit_backward(geo, b.xyz64, b.layer, b.track_hits, r["par"], r["cov"], 1e4)
    ok = (r["status"] == 0) & (rb["status"] == 0)
    truth = b.true_state[:, _first_hits(b)][:, ok]
    for i, pull in _pulls(rb["par"][:, ok], truth, rb["cov"][:, ok]).items():
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i


def test_find_in_parameterised_field_clean_events():
    """No noise, no inefficiency: finding in the parameterised field recovers
    every seed's particle hits exactly."""
    b = make_batch("fit10", [7], n_tracks=300, ineff=0.0, field_alpha=ALPHA)
    geo = O.geometry_for(b)
    for nb in (1, 10):
        r = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=nb)
        for t in range(b.n_seeds):
            want = set(b.track_hits[:, t][b.track_hits[:, t] >= 0])
            got = set(r["hits"][:, t][r["hits"][:, t] >= 0])
            assert got == want, t


def test_rk_from_hit_to_hit_including_grazing_crossings():
    """Every step between consecutive crossings of tracks the generator moved
    through the field (its crossings agree with DOP853, above): from the true
    state at one crossing the oracle lands on the generator's next crossing
    within its truncation error, grazing crossings included (the track meeting
    the cylinder at a few degrees, near its largest radius)."""
    b = make_batch("fit10", [31, 33], n_tracks=400, field_alpha=ALPHA, smear=False)
    geo = O.geometry_for(b)
    grazing = 0
    for t in range(b.n_seeds):
        hh = b.track_hits[:, t]
        hh = hh[hh >= 0]
        for h0, h1 in zip(hh[:-1], hh[1:]):
            r = O.propagate(geo, b.true_state[:, h0], b.layer[h1])
            assert r is not None
            q, want = r[0], b.true_state[:, h1]
            d = q - want
            d[4] = wrap(d[4])
            assert np.abs(d[:3]).max() < TOL_POS, (t, h1, d)
            assert abs(d[3]) < TOL_ANG * abs(want[3]) and np.abs(d[4:]).max() < TOL_ANG, (t, h1, d)
            radial = np.sin(want[5]) * np.cos(want[4] - np.arctan2(want[1], want[0]))
            grazing += radial < 0.15
    assert grazing >= 2


def test_fit_in_parameterised_field_with_disks_pulls():
    """find20 (5 disks per side up to |z| = 270 cm) moved through the field:
    the fit's pulls are N(0, 1) there too; the uniform-field filter's chi2/ndf
    is off on the same hits."""
    alpha = 3e-6
    b = make_batch("find20", [0, 1], n_tracks=1500, field_alpha=alpha)
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    ok = r["status"] == 0
    assert ok.mean() > 0.99
    truth = b.true_state[:, _last_hits(b)][:, ok]
    # q/pT, phi, theta (many tracks end on a disk, where z is fixed)
    for i, pull in _pulls(r["par"][:, ok], truth, r["cov"][:, ok], (3, 4, 5)).items():
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i
    assert abs(r["chi2"][ok].sum() / r["ndf"][ok].sum() - 1) < 0.03
    r0 = O.fit(O.Geometry(b.layers, b.bz), b.xyz64, b.layer, b.track_hits)
    assert r0["chi2"][ok].sum() / r0["ndf"][ok].sum() > 2
