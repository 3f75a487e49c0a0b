"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks an oracle function against something the oracle does not
compute itself: the generator's crossings (closed form from the beam line),
closed forms from the origin, finite differences, the composition law of
Jacobians, limits of the Kalman update, the information form, the Joseph form,
an independent global least-squares helix fit (scipy), brute-force enumeration
of candidate trees, and statistical properties (pulls, chi2/ndf).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from synth import K_FIELD, make_batch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


@pytest.fixture(scope="module")
def find20():
    b = make_batch("find20", [0], n_tracks=400)
    return b, O.geometry_for(b)


# --------------------------------------------------------------------------
# propagation
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cfg", ["find20", "fit10_b0", "dense45"])
def test_propagation_lands_on_generator_crossings(cfg):
    """Propagating the true state at hit k to the layer of hit k+1 reproduces the
    generator's crossing (closed form from the beam line) and its true direction."""
    b = make_batch(cfg, [3], n_tracks=300, smear=False)
    geo = O.geometry_for(b)
    worst_pos, worst_phi, n = 0.0, 0.0, 0
    for t in range(b.n_seeds):
        hh = b.track_hits[:, t]
        hh = hh[hh >= 0]
        for a, c in zip(hh[:-1], hh[1:]):
            res = O.propagate(geo, b.true_state[:, a], b.layer[c])
            assert res is not None
            q, _, s = res
            assert s > 0
            worst_pos = max(worst_pos, np.abs(q[:3] - b.true_xyz[:, c]).max())
            worst_phi = max(worst_phi, abs(wrap(q[4] - b.true_state[4, c])))
            n += 1
    assert n > 500
    assert worst_pos < 1e-8
    assert worst_phi < 1e-10


def test_golden_closed_forms():
    """Textbook closed forms from the origin: radius of curvature pT/(K B), path
    to radius R is 2 rho asin(R / 2 rho), the direction turns by twice the
    position angle, z grows by s cot(theta)."""
    with open(os.path.join(GOLDEN, "helix_closed_forms.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        lay = [dict(kind=0, r_or_z=c["R"], lo=-1e4, hi=1e4, sigma_u=1e-3, sigma_v=1e-3, n_phi=1, n_zr=1)]
        geo = O.Geometry(lay, c["bz"])
        p = np.array([0.0, 0.0, c["z0"], c["q"] / c["pt"], c["phi0"], c["theta"]])
        q, _, s = O.propagate(geo, p, 0)
        assert abs(s - c["s"]) < 1e-9 * c["s"]
        assert np.allclose(q[:3], c["xyz"], atol=1e-9)
        assert abs(wrap(q[4] - c["phi"])) < 1e-12


def test_closed_form_from_origin_random():
    rng = np.random.default_rng(7)
    for _ in range(200):
        pt, q = rng.uniform(0.5, 20), rng.choice([-1.0, 1.0])
        bz, R = 3.8, rng.uniform(2, 60)
        rho = pt / (K_FIELD * bz)
        if R > 2 * rho:
            continue
        phi0, theta = rng.uniform(-np.pi, np.pi), rng.uniform(0.3, 2.8)
        geo = O.Geometry([dict(kind=0, r_or_z=R, lo=-1e4, hi=1e4, sigma_u=1, sigma_v=1)], bz)
        out = O.propagate(geo, [0, 0, 0.5, q / pt, phi0, theta], 0)
        a = math.asin(R / (2 * rho))
        turn = -q  # positive charge turns clockwise in +Bz
        assert abs(out[2] - 2 * rho * a) < 1e-9
        assert abs(wrap(out[0][4] - (phi0 + turn * 2 * a))) < 1e-11
        assert abs(wrap(math.atan2(out[0][1], out[0][0]) - (phi0 + turn * a))) < 1e-11
        assert abs(out[0][2] - (0.5 + 2 * rho * a / math.tan(theta))) < 1e-9


def test_reverse_round_trip(find20):
    """Reversing the direction of motion (phi+pi, theta -> pi-theta, charge flipped)
    and propagating back returns to the start point."""
    b, geo = find20
    worst = 0
    for t in range(100):
        a, c = b.track_hits[0, t], b.track_hits[2, t]
        p0 = b.true_state[:, a]
        q, _, _ = O.propagate(geo, p0, b.layer[c])
        rev = np.array([q[0], q[1], q[2], -q[3], wrap(q[4] + np.pi), np.pi - q[5]])
        back = O.propagate(geo, rev, b.layer[a])
        assert back is not None
        worst = max(worst, np.abs(back[0][:3] - p0[:3]).max())
        assert abs(wrap(back[0][4] - wrap(p0[4] + np.pi))) < 1e-11
    assert worst < 1e-9


def test_straight_line_limit():
    """B = 0: the crossing with radius R from (x, y) along phi solves |P + s u| = R."""
    rng = np.random.default_rng(3)
    geo = O.Geometry([dict(kind=0, r_or_z=50.0, lo=-1e4, hi=1e4, sigma_u=1, sigma_v=1)], 0.0)
    for _ in range(100):
        x, y = rng.uniform(-20, 20, 2)
        phi = rng.uniform(-np.pi, np.pi)
        q, _, s = O.propagate(geo, [x, y, 0, 0.3, phi, 1.0], 0)
        assert abs(math.hypot(q[0], q[1]) - 50.0) < 1e-10
        assert abs(q[0] - (x + s * math.cos(phi))) < 1e-10 and abs(q[1] - (y + s * math.sin(phi))) < 1e-10
        assert q[4] == pytest.approx(phi)


def test_unreachable_layers():
    geo = O.Geometry([dict(kind=0, r_or_z=200.0, lo=-1e4, hi=1e4, sigma_u=1, sigma_v=1),
                      dict(kind=1, r_or_z=-50.0, lo=0, hi=1e4, sigma_u=1, sigma_v=1)], 3.8)
    # pT = 0.5 GeV: 2 rho = 87.8 cm < 200 cm
    assert O.propagate(geo, [0, 0, 0, 1 / 0.5, 0.1, 1.0], 0) is None
    # disk behind the track
    assert O.propagate(geo, [0, 0, 0, 1 / 2.0, 0.1, 1.0], 1) is None


# --------------------------------------------------------------------------
# Jacobian and transport
# --------------------------------------------------------------------------

def _fd_jacobian(geo, p, l, rel=1e-6):
    J = np.zeros((6, 6))
    for j in range(6):
        h = rel * max(1.0, abs(p[j]))

        def f(dv):
            pp = np.array(p, dtype=float)
            pp[j] += dv
            return O.propagate(geo, pp, l)[0]

        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
        J[:, j] = (4 * d1 - d2) / 3
    return J


@pytest.mark.parametrize("cfg", ["find20", "fit10_b0"])
def test_jacobian_matches_finite_differences(cfg):
    b = make_batch(cfg, [1], n_tracks=150, smear=False)
    geo = O.geometry_for(b)
    kinds = set()
    worst = 0
    for t in range(b.n_seeds):
        a, c = b.seed_hits[0, t], b.seed_hits[2, t]
        p = b.true_state[:, a]
        q, J, _ = O.propagate(geo, p, b.layer[c])
        Jfd = _fd_jacobian(geo, p, b.layer[c])
        worst = max(worst, np.abs(J - Jfd).max() / max(1.0, np.abs(J).max()))
        kinds.add(int(geo.kind[b.layer[c]]))
    assert worst < 1e-6
    if cfg == "find20":
        assert kinds == {0, 1}


def test_jacobian_chain_rule(find20):
    b, geo = find20
    for t in range(50):
        hh = b.track_hits[:, t]
        hh = hh[hh >= 0]
        pa = b.true_state[:, hh[0]]
        qb, Jab, _ = O.propagate(geo, pa, b.layer[hh[1]])
        qc, Jbc, _ = O.propagate(geo, qb, b.layer[hh[2]])
        qc2, Jac, _ = O.propagate(geo, pa, b.layer[hh[2]])
        assert np.allclose(qc[:3], qc2[:3], atol=1e-9)
        assert np.allclose(Jbc @ Jab, Jac, rtol=1e-7, atol=1e-9)


def test_transport_symmetric_psd_and_normal_variance(find20):
    b, geo = find20
    rng = np.random.default_rng(5)
    for t in range(60):
        a, c = b.seed_hits[0, t], b.seed_hits[2, t]
        q, J, _ = O.propagate(geo, b.true_state[:, a], b.layer[c])
        A = rng.normal(size=(6, 6))
        C0 = A @ A.T * 1e-3 + np.eye(6) * 1e-5
        C1 = O.transport(J, C0)
        assert np.allclose(C1, C1.T)
        assert np.allclose(C1, J @ C0 @ J.T, rtol=1e-12, atol=1e-15)
        assert np.linalg.eigvalsh(C1).min() > -1e-12 * np.abs(C1).max()
        l = b.layer[c]
        if geo.kind[l] == 0:
            n = np.array([q[0], q[1], 0, 0, 0, 0]) / math.hypot(q[0], q[1])
        else:
            n = np.array([0, 0, 1.0, 0, 0, 0])
        assert n @ C1 @ n < 1e-10 * np.trace(C1)


# --------------------------------------------------------------------------
# Kalman update
# --------------------------------------------------------------------------

def _setup_update(seed=0, kind=0, dphi=2e-5):
    rng = np.random.default_rng(seed)
    if kind == 0:
        lay = [dict(kind=0, r_or_z=30.0, lo=-100, hi=100, sigma_u=0.002, sigma_v=0.01)]
        phi = rng.uniform(-np.pi, np.pi)
        p = np.array([30 * math.cos(phi), 30 * math.sin(phi), 5.0, 0.4, phi + 0.1, 1.2])
        hit = np.array([30 * math.cos(phi + dphi), 30 * math.sin(phi + dphi), 5.0 + 100 * dphi])
    else:
        lay = [dict(kind=1, r_or_z=120.0, lo=5, hi=100, sigma_u=0.002, sigma_v=0.01)]
        phi = rng.uniform(-np.pi, np.pi)
        p = np.array([40 * math.cos(phi), 40 * math.sin(phi), 120.0, 0.4, phi + 0.1, 0.4])
        hit = np.array([(40 + 50 * dphi) * math.cos(phi + dphi), (40 + 50 * dphi) * math.sin(phi + dphi), 120.0])
    A = rng.normal(size=(6, 6))
    Cm = A @ A.T * 1e-4 + np.eye(6) * 1e-4
    return lay, p, Cm, hit


@pytest.mark.parametrize("kind", [0, 1])
def test_update_limits(kind):
    lay, p, Cm, hit = _setup_update(1, kind)
    # a transported covariance has no variance along the surface normal
    n = np.zeros(6)
    if kind == 0:
        n[:2] = p[:2] / math.hypot(p[0], p[1])
    else:
        n[2] = 1.0
    P = np.eye(6) - np.outer(n, n)
    Cm = P @ Cm @ P
    # V -> 0: the updated position reproduces the hit (up to the curvature of
    # the surface coordinates: second order in the residual)
    lay0 = [dict(lay[0], sigma_u=1e-9, sigma_v=1e-9)]
    p1, C1, chi2, r, S, _ = O.update(O.Geometry(lay0, 3.8), 0, hit, p, Cm)
    _, _, _, r_after, _, _ = O.update(O.Geometry(lay0, 3.8), 0, hit, p1, C1)
    second_order = np.abs(r).max() ** 2 / math.hypot(p[0], p[1])
    assert np.abs(r_after).max() < 2 * second_order + 1e-9
    # V -> infinity: nothing moves, chi2 -> 0
    layi = [dict(lay[0], sigma_u=1e6, sigma_v=1e6)]
    p2, C2, chi2i, _, _, _ = O.update(O.Geometry(layi, 3.8), 0, hit, p, Cm)
    assert np.allclose(p2, p, atol=1e-9) and np.allclose(C2, Cm, atol=1e-12) and chi2i < 1e-10


@pytest.mark.parametrize("kind", [0, 1])
def test_update_information_form_and_joseph(kind):
    # a small residual: the r-phi lever arm's own dependence on x, y (left out of
    # H by definition) is then below the tolerances
    lay, p, Cm, hit = _setup_update(2, kind, dphi=1e-7)
    geo = O.Geometry(lay, 3.8)
    p1, C1, chi2, r, S, Cj = O.update(geo, 0, hit, p, Cm)
    # H as the derivative of the residual's prediction: numerically from the residual itself
    H = np.zeros((2, 6))
    for j in range(3):
        d = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[j] += d
        pm[j] -= d
        rp = O.update(geo, 0, hit, pp, Cm)[3]
        rm = O.update(geo, 0, hit, pm, Cm)[3]
        H[:, j] = -(rp - rm) / (2 * d)
    V = np.diag([lay[0]["sigma_u"] ** 2, lay[0]["sigma_v"] ** 2])
    # the oracle's H drops the (tiny) dependence of the r-phi lever arm on x, y
    assert np.allclose(S, H @ Cm @ H.T + V, rtol=1e-5)
    info = np.linalg.inv(Cm) + H.T @ np.linalg.inv(V) @ H
    assert np.allclose(np.linalg.inv(C1), info, rtol=1e-4, atol=1e-6 * np.abs(info).max())
    assert np.allclose(C1, Cj, rtol=1e-9, atol=1e-14)
    assert chi2 == pytest.approx(r @ np.linalg.solve(S, r), rel=1e-12)
    # p1 - p = C1 H^T V^-1 r  (gain in information form)
    assert np.allclose(p1 - p, C1 @ H.T @ np.linalg.solve(V, r), rtol=1e-4, atol=1e-10)


# --------------------------------------------------------------------------
# seeds and fit
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cfg", ["find20", "fit10_b0"])
def test_seed_exact_on_noise_free_helix(cfg):
    b = make_batch(cfg, [2], n_tracks=200, smear=False)
    geo = O.geometry_for(b)
    for t in range(b.n_seeds):
        h = b.seed_hits[:, t]
        p, _ = O.seed(geo, b.xyz64[:, h[0]], b.xyz64[:, h[1]], b.xyz64[:, h[2]], b.layer[h[0]])
        ts = b.true_state[:, h[0]]
        assert np.allclose(p[:3], ts[:3], atol=1e-9)
        assert abs(wrap(p[4] - ts[4])) < 1e-8
        assert abs(p[5] - ts[5]) < 1e-8
        if b.bz != 0:
            assert abs(p[3] - ts[3]) < 1e-8 * max(1, abs(ts[3]))


def _last_hits(b):
    out = []
    for t in range(b.n_seeds):
        hh = b.track_hits[:, t]
        out.append(hh[hh >= 0][-1])
    return np.array(out)


def test_fit_noise_free_recovers_truth():
    for cfg in ["fit10", "fit10_b0", "find20"]:
        b = make_batch(cfg, [4], n_tracks=300, smear=False)
        geo = O.geometry_for(b)
        r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
        ts = b.true_state[:, _last_hits(b)]
        d = r["par"] - ts
        d[4] = wrap(d[4])
        if b.bz == 0:
            d[3] = 0
        scale = np.maximum(1.0, np.abs(ts))
        assert np.abs(d / scale).max() < 1e-9
        assert r["chi2"].max() < 1e-12
        assert (r["status"] == 0).all()


@pytest.mark.slow
def test_fit_pulls_and_chi2():
    b = make_batch("fit10", list(range(10)))
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    ts = b.true_state[:, _last_hits(b)]
    Cm = O.unpack21(r["cov"])
    for i in range(6):
        d = r["par"][i] - ts[i]
        if i == 4:
            d = wrap(d)
        pull = d / np.sqrt(Cm[:, i, i])
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i
    assert abs(r["chi2"].sum() / r["ndf"].sum() - 1) < 0.03
    # chi2 probability is flat: deciles of the chi2 CDF
    from scipy.stats import chi2 as chi2d
    pr = chi2d.sf(r["chi2"], r["ndf"])
    hist = np.histogram(pr, bins=10, range=(0, 1))[0] / pr.size
    assert np.abs(hist - 0.1).max() < 0.025


def test_fit_prior_inflation_negligible():
    b = make_batch("fit10", [5], n_tracks=300)
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    # seeds from the same 3 hits, prior covariance inflated x10 in variance
    sp, sc = [], []
    for t in range(b.n_seeds):
        h = b.track_hits[:3, t]
        p, Cm = O.seed(geo, b.xyz64[:, h[0]], b.xyz64[:, h[1]], b.xyz64[:, h[2]], b.layer[h[0]])
        sp.append(p)
        sc.append(Cm * 10.0)
    r10 = O.fit(geo, b.xyz64, b.layer, b.track_hits, np.array(sp).T, O.pack21(np.array(sc)))
    Cm = O.unpack21(r["cov"])
    for i in range(6):
        d = r10["par"][i] - r["par"][i]
        if i == 4:
            d = wrap(d)
        assert np.abs(d / np.sqrt(Cm[:, i, i])).max() < 0.05, i


def _global_ls(geo, b, t):
    """Independent global least-squares helix fit through the track's hits:
    5 parameters (azimuth of the start on the first cylinder, z, q/pT, phi,
    theta), crossings by root finding on the closed-form helix."""
    import scipy.optimize as so
    hh = b.track_hits[:, t]
    hh = hh[hh >= 0]
    Hx = b.xyz64[:, hh].T
    R = np.array([geo.rz[b.layer[i]] for i in hh])
    su, sv = geo.su[b.layer[hh]], geo.sv[b.layer[hh]]

    def path(a, z0, w, phi, th):
        x0, y0 = R[0] * math.cos(a), R[0] * math.sin(a)
        h = -w * K_FIELD * b.bz
        pts = [(x0, y0, z0, phi)]
        for Rk in R[1:]:
            f = lambda s: math.hypot(x0 + (math.sin(phi + h * s) - math.sin(phi)) / h,
                                     y0 - (math.cos(phi + h * s) - math.cos(phi)) / h) - Rk
            s = so.brentq(f, 1e-9, math.pi / abs(h) * (1 - 1e-12), xtol=1e-14)
            pts.append((x0 + (math.sin(phi + h * s) - math.sin(phi)) / h,
                        y0 - (math.cos(phi + h * s) - math.cos(phi)) / h, z0 + s / math.tan(th), phi + h * s))
        return np.array(pts)

    def resid(v):
        P = path(*v)
        u = R * wrap(np.arctan2(Hx[:, 1], Hx[:, 0]) - np.arctan2(P[:, 1], P[:, 0]))
        return np.concatenate([u / su, (Hx[:, 2] - P[:, 2]) / sv])

    ts = b.true_state[:, hh[0]]
    v0 = [math.atan2(ts[1], ts[0]), ts[2], ts[3], ts[4], ts[5]]
    sol = so.least_squares(resid, v0, x_scale="jac", xtol=1e-14, ftol=1e-14, gtol=1e-14)
    P = path(*sol.x)
    last = np.array([P[-1, 0], P[-1, 1], P[-1, 2], sol.x[2], wrap(P[-1, 3]), sol.x[4]])
    first = np.array([P[0, 0], P[0, 1], P[0, 2], sol.x[2], wrap(P[0, 3]), sol.x[4]])
    return (sol.fun ** 2).sum(), last, first


def test_fit_matches_global_least_squares():
    b = make_batch("fit10", [6], n_tracks=40)
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    Cm = O.unpack21(r["cov"])
    for t in range(b.n_seeds):
        if b.particle_nhits[b.seed_particle[t]] < 10:
            continue
        chi2_ls, last, _ = _global_ls(geo, b, t)
        d = r["par"][:, t] - last
        d[4] = wrap(d[4])
        assert np.abs(d / np.sqrt(np.diag(Cm[t]))).max() < 0.05, t
        assert abs(r["chi2"][t] - chi2_ls) < 0.05 * max(1.0, chi2_ls), t


# --------------------------------------------------------------------------
# backward fit
# --------------------------------------------------------------------------

def _first_hits(b):
    return np.array([b.track_hits[:, t][b.track_hits[:, t] >= 0][0] for t in range(b.n_seeds)])


def test_backfit_noise_free_recovers_truth():
    """Noise-free hits: the backward pass from the forward result returns the
    generator's state at each track's first hit, whatever the inflation."""
    for cfg in ["fit10", "fit10_b0", "find20", "dense45"]:
        b = make_batch(cfg, [4], n_tracks=200, smear=False)
        geo = O.geometry_for(b)
        r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
        ok = r["status"] == 0
        ts = b.true_state[:, _first_hits(b)]
        for inflate in (1.0, 100.0, 1e4):
            rb = O.fit_backward(geo, b.xyz64, b.layer, b.track_hits, r["par"], r["cov"], inflate)
            assert (rb["status"][ok] == 0).all(), cfg
            d = rb["par"][:, ok] - ts[:, ok]
            d[4] = wrap(d[4])
            if b.bz == 0:
                d[3] = 0
            scale = np.maximum(1.0, np.abs(ts[:, ok]))
            assert np.abs(d / scale).max() < 1e-9, (cfg, inflate)
            assert rb["chi2"][ok].max() < 1e-12
            assert (rb["ndf"][ok] == r["ndf"][ok]).all()


@pytest.mark.slow
def test_backfit_pulls_and_chi2():
    """Smeared hits: pulls of the state at the first hit against the generator
    are N(0, 1) and chi2/ndf is 1 (a sign error in the turned-around covariance
    or transport shows in both)."""
    b = make_batch("find20", list(range(3)), n_tracks=1500)
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    rb = O.fit_backward(geo, b.xyz64, b.layer, b.track_hits, r["par"], r["cov"], 1e4)
    ok = (rb["status"] == 0) & (r["status"] == 0)
    first = _first_hits(b)
    assert (geo.kind[b.layer[first]] == 0).all()  # every track starts on a cylinder
    ts = b.true_state[:, first]
    Cm = O.unpack21(rb["cov"][:, ok])
    # position along the surface (r-phi): x and y alone mix in the radial
    # direction, whose variance on the surface is zero to first order
    phi_pos = np.arctan2(ts[1, ok], ts[0, ok])
    hu = np.zeros((ok.sum(), 6))
    hu[:, 0], hu[:, 1] = -np.sin(phi_pos), np.cos(phi_pos)
    du = hu[:, 0] * (rb["par"][0, ok] - ts[0, ok]) + hu[:, 1] * (rb["par"][1, ok] - ts[1, ok])
    pulls = {"u": du / np.sqrt(np.einsum("ti,tij,tj->t", hu, Cm, hu))}
    for i in range(2, 6):
        d = rb["par"][i, ok] - ts[i, ok]
        if i == 4:
            d = wrap(d)
        pulls[i] = d / np.sqrt(Cm[:, i, i])
    for k, pull in pulls.items():
        assert abs(pull.mean()) < 0.05, k
        assert abs(pull.std() - 1) < 0.05, k
    assert abs(rb["chi2"][ok].sum() / rb["ndf"][ok].sum() - 1) < 0.03


def test_backfit_matches_global_least_squares():
    """With a vague prior (inflation 1e4) the backward pass is the least-squares
    helix through all the hits, reported at the first hit: state and chi2 agree
    with an independent global fit (scipy)."""
    b = make_batch("fit10", [6], n_tracks=40)
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    rb = O.fit_backward(geo, b.xyz64, b.layer, b.track_hits, r["par"], r["cov"], 1e4)
    Cm = O.unpack21(rb["cov"])
    n_checked = 0
    for t in range(b.n_seeds):
        if b.particle_nhits[b.seed_particle[t]] < 10:
            continue
        chi2_ls, _, first = _global_ls(geo, b, t)
        d = rb["par"][:, t] - first
        d[4] = wrap(d[4])
        assert np.abs(d / np.sqrt(np.diag(Cm[t]))).max() < 0.05, t
        assert abs(rb["chi2"][t] - chi2_ls) < 0.05 * max(1.0, chi2_ls), t
        n_checked += 1
    assert n_checked >= 20


@pytest.mark.parametrize("cfg", ["fit10", "find20"])
def test_backfit_transport_round_trip(cfg):
    """With hit errors of 1e4 cm the updates do nothing measurable, so the
    backward pass only carries the state and covariance from the last hit back
    to the first: it must return the first-hit state and the on-surface
    covariance that the forward Jacobians (or_propagate, or_transport) carried
    from the first hit to the last.  A wrong sign in the turned-around
    covariance, or a transport that does not invert, fails here."""
    b = make_batch(cfg, [8], n_tracks=60, smear=False)
    geo = O.geometry_for(b)
    big = O.Geometry([dict(d, sigma_u=1e4, sigma_v=1e4) for d in b.layers], b.bz)
    lp, lc, p0s, c0s = [], [], [], []
    for t in range(b.n_seeds):
        hh = b.track_hits[:, t]
        hh = hh[hh >= 0]
        p, Cm = O.seed(geo, *[b.xyz64[:, i] for i in hh[:3]], b.layer[hh[0]])
        p = b.true_state[:, hh[0]].copy()
        p0s.append(p.copy())
        c0s.append(Cm.copy())
        for h in hh[1:]:
            q, J, _ = O.propagate(geo, p, b.layer[h])
            Cm = O.transport(J, Cm)
            p = q
        lp.append(p)
        lc.append(Cm)
    rb = O.fit_backward(big, b.xyz64, b.layer, b.track_hits, np.array(lp).T, O.pack21(np.array(lc)), 1.0)
    assert (rb["status"] == 0).all()
    d = rb["par"] - np.array(p0s).T
    d[4] = wrap(d[4])
    assert np.abs(d).max() < 1e-9
    Cb = O.unpack21(rb["cov"])
    C0 = np.array(c0s)
    sd = np.sqrt(np.einsum("tii->ti", C0))
    assert (np.abs(Cb - C0) / (sd[:, :, None] * sd[:, None, :] + 1e-300)).max() < 1e-5


def test_backfit_short_lists_and_errors():
    b = make_batch("fit10", [7], n_tracks=20)
    geo = O.geometry_for(b)
    hidx = b.track_hits.copy()
    hidx[2:, 3] = -1  # two hits: no fit
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    rb = O.fit_backward(geo, b.xyz64, b.layer, hidx, r["par"], r["cov"], 100.0)
    assert rb["status"][3] & 2 and np.isnan(rb["par"][:, 3]).all()
    with pytest.raises(RuntimeError):
        O.fit_backward(geo, b.xyz64, b.layer, hidx, r["par"], r["cov"], 0.5)


# --------------------------------------------------------------------------
# material: multiple scattering
# --------------------------------------------------------------------------

def _chi2_median_over_ndf(ndf):
    """Mean over tracks of the median of chi2(ndf) / ndf (what the median of
    chi2 / ndf is for a correct fit)."""
    from scipy.stats import chi2 as chi2_dist
    return float(np.median(chi2_dist.rvs(ndf, random_state=np.random.default_rng(0)) / ndf))


def _pulls(par, truth, cov21, idx=(2, 3, 4, 5)):
    Cm = O.unpack21(cov21)
    out = {}
    for i in idx:
        d = par[i] - truth[i]
        if i == 4:
            d = wrap(d)
        out[i] = d / np.sqrt(Cm[:, i, i])
    return out


@pytest.mark.parametrize("kind", [0, 1])
def test_scattering_noise_is_the_kick_covariance(kind):
    """The noise the oracle adds at a layer equals the covariance of the kick
    model it stands for, sampled: the polar angle and azimuth kicked by theta0
    and theta0 / sin(theta) (theta0 from the generator's Highland function at
    the path through the layer), the momentum magnitude kept, q/pT recomputed
    from it -- which fixes the 1 / sin^2 factor and the q/pT-theta coupling."""
    from synth.events import _highland
    lay = (dict(kind=0, r_or_z=30.0, lo=-100.0, hi=100.0, sigma_u=0.01, sigma_v=0.01, x0=0.05) if kind == 0 else
           dict(kind=1, r_or_z=100.0, lo=5.0, hi=60.0, sigma_u=0.01, sigma_v=0.01, x0=0.05))
    geo = O.Geometry([lay], 3.8)
    rng = np.random.default_rng(11 + kind)
    for p in ([30 * math.cos(0.4), 30 * math.sin(0.4), 10.0, 0.7, 0.7, 0.55],
              [21.0, 9.0, 100.0, -1.6, -2.9, 0.35] if kind else [-12.0, 27.4955, -40.0, -1.6, 1.4, 2.3]):
        p = np.array(p)
        if kind == 0:
            p[:2] *= 30.0 / math.hypot(p[0], p[1])
        Q = O.scattering(geo, 0, p)
        st = math.sin(p[5])
        cosa = abs(st * math.cos(p[4] - math.atan2(p[1], p[0]))) if kind == 0 else abs(math.cos(p[5]))
        pm = 1.0 / (abs(p[3]) * st)
        t0 = float(_highland(pm, 0.05 / cosa))
        g = rng.standard_normal((2, 2_000_000))
        dth = t0 * g[0]
        dphi = t0 * g[1] / st
        dw = np.sign(p[3]) / (pm * np.sin(p[5] + dth)) - p[3]
        S = np.cov(np.stack([dw, dphi, dth]))
        q = Q[3:, 3:]
        for i in range(3):
            assert abs(S[i, i] / q[i, i] - 1) < 0.01, (i, S[i, i], q[i, i])
        assert abs(S[0, 2] / q[0, 2] - 1) < 0.02
        assert abs(q[0, 1]) == 0 and abs(q[1, 2]) == 0 and abs(S[0, 1]) < 0.01 * math.sqrt(S[0, 0] * S[1, 1])
        assert (Q[:3] == 0).all() and (Q[:, :3] == 0).all()


def test_fit_with_scattering_pulls_and_chi2():
    """Tracks that scatter in 0.03 X0 per layer (the generator moves them layer
    by layer with Gaussian kicks): with the scattering noise the fit's pulls at
    the last hit are N(0, 1) and chi2/ndf is 1; without it chi2/ndf is far above
    1 (the test has the power to see a wrong noise)."""
    b = make_batch("fit10", list(range(6)), n_tracks=1000, material=0.03)
    geo = O.geometry_for(b)
    assert (geo.x0 == 0.03).all()
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    ok = r["status"] == 0
    assert ok.mean() > 0.99
    for i, pull in _pulls(r["par"][:, ok], b.true_state[:, _last_hits(b)][:, ok], r["cov"][:, ok]).items():
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i
    assert abs(r["chi2"][ok].sum() / r["ndf"][ok].sum() - 1) < 0.03
    bare = O.Geometry([{k: v for k, v in d.items() if k != "x0"} for d in b.layers], b.bz)
    r0 = O.fit(bare, b.xyz64, b.layer, b.track_hits)
    assert r0["chi2"][ok].sum() / r0["ndf"][ok].sum() > 5


def test_fit_with_energy_loss_pulls():
    """Tracks that also lose energy (0.15 GeV per X0, exaggerated so that the
    loss is several q/pT sigmas over the track): with the mean loss in the
    filter the q/pT pull at the last hit is N(0, 1); without it the pull widens
    past 1.5."""
    b = make_batch("fit10", list(range(6)), n_tracks=1000, material=0.03, eloss=0.15)
    geo = O.geometry_for(b)
    assert (geo.eloss == 0.15).all()
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    ok = r["status"] == 0
    truth = b.true_state[:, _last_hits(b)][:, ok]
    for i, pull in _pulls(r["par"][:, ok], truth, r["cov"][:, ok]).items():
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i
    assert abs(r["chi2"][ok].sum() / r["ndf"][ok].sum() - 1) < 0.03
    bare = O.Geometry([{k: v for k, v in d.items() if k != "eloss"} for d in b.layers], b.bz)
    r0 = O.fit(bare, b.xyz64, b.layer, b.track_hits)
    assert _pulls(r0["par"][:, ok], truth, r0["cov"][:, ok], (3,))[3].std() > 1.5


def test_fit_with_material_on_cylinders_and_disks():
    """The dense layout (17 cylinders + 2 x 14 disks) with 0.02 X0 and 0.04 GeV
    per X0 in every layer: the generator moves the particles from surface to
    surface in path order, kicking and slowing them at every layer crossed
    (on a disk the path through it is x0 / |cos(theta)|); with the material
    in the filter the pulls of q/pT, phi and theta at the last hit are N(0, 1)
    and chi2/ndf is 1, without it chi2/ndf is far off."""
    b = make_batch("dense45", [3, 4], n_tracks=1200, n_noise=0, material=0.02, eloss=0.04)
    disk = np.array([d["kind"] for d in b.layers])[b.layer] == 1
    assert disk[b.hit_particle >= 0].mean() > 0.2  # many hits on disks
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    ok = r["status"] == 0
    assert ok.mean() > 0.99
    truth = b.true_state[:, _last_hits(b)][:, ok]
    # widths from the median absolute deviation: a few low-pT particles that
    # lose most of their energy in the 45 layers leave the Gaussian regime
    # (two of 2400 with |pull| > 6), which the standard deviation would weigh
    for i, pull in _pulls(r["par"][:, ok], truth, r["cov"][:, ok], (3, 4, 5)).items():
        med = np.median(pull)
        assert abs(med) < 0.05, i
        assert abs(1.4826 * np.median(np.abs(pull - med)) - 1) < 0.05, i
        assert (np.abs(pull) > 6).mean() < 3e-3, i
    assert abs(np.median(r["chi2"][ok] / r["ndf"][ok]) / _chi2_median_over_ndf(r["ndf"][ok]) - 1) < 0.05
    bare = O.Geometry([{k: v for k, v in d.items() if k not in ("x0", "eloss")} for d in b.layers], b.bz)
    r0 = O.fit(bare, b.xyz64, b.layer, b.track_hits)
    assert r0["chi2"][ok].sum() / r0["ndf"][ok].sum() > 5


@pytest.mark.parametrize("eloss", [0.0, 0.15])
def test_backfit_with_scattering_pulls_and_chi2(eloss):
    """The backward pass adds each layer's material after its hit (reversed in
    time: the lost energy gained back, then the scattering noise) and ends
    before the first layer's material: its state at the first hit is the
    particle's state there before any scattering or loss -- the vertex direction
    turned by h s and the vertex q/pT and theta."""
    b = make_batch("fit10", list(range(6)), n_tracks=1000, material=0.03, eloss=eloss)
    geo = O.geometry_for(b)
    r = O.fit(geo, b.xyz64, b.layer, b.track_hits)
    rb = O.fit_backward(geo, b.xyz64, b.layer, b.track_hits, r["par"], r["cov"], 1e4)
    ok = (r["status"] == 0) & (rb["status"] == 0)
    first = _first_hits(b)
    pp = b.particle_par[:, b.seed_particle]
    x1, y1 = b.true_xyz[0, first], b.true_xyz[1, first]
    h = -pp[3] * K_FIELD * b.bz
    s1 = 2.0 * np.arcsin(np.hypot(x1, y1) * np.abs(h) / 2.0) / np.abs(h)
    truth = np.stack([x1, y1, b.true_xyz[2, first], pp[3], wrap(pp[4] + h * s1), pp[5]])
    for i, pull in _pulls(rb["par"][:, ok], truth[:, ok], rb["cov"][:, ok]).items():
        assert abs(pull.mean()) < 0.05, i
        assert abs(pull.std() - 1) < 0.05, i
    assert abs(rb["chi2"][ok].sum() / rb["ndf"][ok].sum() - 1) < 0.03


# --------------------------------------------------------------------------
# finding
# --------------------------------------------------------------------------

def test_find_clean_events_full_efficiency():
    """No noise, no inefficiency: every seed recovers exactly its particle's hits."""
    b = make_batch("find20", [7], n_tracks=300, ineff=0.0, noise_scale=0.0)
    geo = O.geometry_for(b)
    for nb in (1, 10):
        r = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=nb)
        for t in range(b.n_seeds):
            want = set(b.track_hits[:, t][b.track_hits[:, t] >= 0])
            got = set(r["hits"][:, t][r["hits"][:, t] >= 0])
            assert got == want, t
        assert (r["n_hits"] == b.particle_nhits[b.seed_particle]).all()


def _enumerate(geo, xyz, layers, ev_hits, seed, cut, max_consec):
    """All leaves of the candidate tree of one seed (tiny events only).

    Restates the finder's rules independently of its beam search: after the
    three-hit seed fit, at every step a candidate goes to its next layer (the
    nearer of the next cylinder and the next disk in path length, layers crossed
    outside their extent passed over), and branches into every compatible hit
    (chi2 < cut) plus one miss; a candidate stops when no layer is left or after
    max_consec consecutive misses."""
    sh = seed
    p, Cm = O.seed(geo, xyz[:, sh[0]], xyz[:, sh[1]], xyz[:, sh[2]], layers[sh[0]])
    chi2 = 0.0
    for k in range(3):
        if k:
            p, J, _ = O.propagate(geo, p, layers[sh[k]])
            Cm = J @ Cm @ J.T
        p, Cm, x2, _, _, _ = O.update(geo, layers[sh[k]], xyz[:, sh[k]], p, Cm)
        chi2 += x2
    cyl = sorted([l for l in range(geo.n) if geo.kind[l] == 0], key=lambda l: geo.rz[l])
    dsk = sorted([l for l in range(geo.n) if geo.kind[l] == 1], key=lambda l: geo.rz[l])
    direction = 1 if math.cos(p[5]) / math.sin(p[5]) >= 0 else -1
    l3 = layers[sh[2]]
    r3, z3 = math.hypot(xyz[0, sh[2]], xyz[1, sh[2]]), xyz[2, sh[2]]
    nc = cyl.index(l3) + 1 if geo.kind[l3] == 0 else next((i for i, l in enumerate(cyl) if geo.rz[l] > r3), len(cyl))
    if geo.kind[l3] == 1:
        nd = dsk.index(l3) + direction
    elif direction > 0:
        nd = next((i for i, l in enumerate(dsk) if geo.rz[l] > z3), len(dsk))
    else:
        nd = next((i for i in range(len(dsk) - 1, -1, -1) if geo.rz[dsk[i]] < z3), -1)
    leaves = []

    def rec(p, Cm, chi2, nh, consec, nc, nd, hits):
        rcur, zcur = math.hypot(p[0], p[1]), p[2]
        while True:
            while 0 <= nc < len(cyl) and geo.rz[cyl[nc]] <= rcur:
                nc += 1
            while 0 <= nd < len(dsk) and direction * (geo.rz[dsk[nd]] - zcur) <= 0:
                nd += direction
            lc = cyl[nc] if 0 <= nc < len(cyl) else None
            ld = dsk[nd] if 0 <= nd < len(dsk) else None
            rc = O.propagate(geo, p, lc) if lc is not None else None
            rd = O.propagate(geo, p, ld) if ld is not None else None
            if rc is None:
                nc = len(cyl)
            if rd is None:
                nd = -1 if direction < 0 else len(dsk)
            if rc is None and rd is None:
                leaves.append((cut * nh - chi2, hits))
                return
            use_c = rd is None or (rc is not None and rc[2] <= rd[2])
            l, (q, J, _) = (lc, rc) if use_c else (ld, rd)
            if use_c:
                nc += 1
            else:
                nd += direction
            coord = q[2] if geo.kind[l] == 0 else math.hypot(q[0], q[1])
            if geo.lo[l] <= coord <= geo.hi[l]:
                break
        Cq = J @ Cm @ J.T
        for hid in ev_hits[l]:
            p2, C2, x2, _, _, _ = O.update(geo, l, xyz[:, hid], q, Cq)
            if x2 < cut:
                rec(p2, C2, chi2 + x2, nh + 1, 0, nc, nd, hits + [hid])
        if consec + 1 >= max_consec:
            leaves.append((cut * nh - chi2, hits))
        else:
            rec(q, Cq, chi2, nh, consec + 1, nc, nd, hits)

    rec(p, Cm, chi2, 3, 0, nc, nd, [])
    return leaves


def test_find_brute_force_tiny_events():
    """Tiny events (3 tracks, 10 noise hits per layer) on a 5-layer detector:
    N-best with N larger than the tree width returns the best leaf of the
    exhaustive enumeration; best-hit finding never scores above it."""
    lay = [dict(kind=0, r_or_z=r, lo=-60, hi=60, sigma_u=0.05, sigma_v=0.2, n_phi=4, n_zr=2)
           for r in (4.0, 9.0, 15.0, 22.0, 30.0)]
    from synth import configs as cf
    cf.CONFIGS["_tiny"] = dict(layers=lay, bz=3.8, n_tracks=3, eta_max=0.8, pt_min=0.8, pt_max=3.0,
                               pt_spectrum="flat", z0_half=2.0, ineff=0.1, noise_mode="total", noise=50)
    cf.CONFIG_IDS["_tiny"] = 99
    try:
        checked = 0
        for ev in range(12):
            b = make_batch("_tiny", [ev])
            geo = O.geometry_for(b)
            xyz = b.xyz.astype(np.float64)
            ev_hits = {l: list(np.nonzero(b.layer == l)[0]) for l in range(geo.n)}
            for t in range(b.n_seeds):
                leaves = _enumerate(geo, xyz, b.layer, ev_hits, b.seed_hits[:, t], 30.0, 3)
                best = max(s for s, _ in leaves)
                rn = O.find(geo, xyz, b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=16,
                            seed_list=[t], max_out=8)
                r1 = O.find(geo, xyz, b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=1,
                            seed_list=[t], max_out=8)
                sn = 30.0 * rn["n_hits"][0] - rn["chi2"][0]
                s1 = 30.0 * r1["n_hits"][0] - r1["chi2"][0]
                assert s1 <= sn + 1e-9
                if len(leaves) <= 16:
                    assert sn == pytest.approx(best, abs=1e-9)
                    got = list(rn["hits"][3:, 0][rn["hits"][3:, 0] >= 0])
                    assert any(sorted(h) == sorted(got) and abs(s - best) < 1e-9 for s, h in leaves)
                    checked += 1
        assert checked >= 20
    finally:
        cf.CONFIGS.pop("_tiny")
        cf.CONFIG_IDS.pop("_tiny")


def test_find_region_masks_restrict_layers(find20):
    b, _ = find20
    n = len(b.layers)
    allmask = (1 << n) - 1
    odd_cyl = sum(1 << l for l in range(n) if b.layers[l]["kind"] == 0 and l % 2 == 1)
    geo = O.Geometry(b.layers, b.bz, region_edges=[-0.9, 0.9], region_masks=[allmask, allmask & ~odd_cyl, allmask])
    r = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=1)
    geo_all = O.geometry_for(b)
    r_all = O.find(geo_all, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=1)
    changed = 0
    for t in range(b.n_seeds):
        found = r["hits"][3:, t]
        found = found[found >= 0]
        barrel_region = abs(np.arcsinh(1 / math.tan(b.true_state[5, b.seed_hits[0, t]]))) < 0.85
        if barrel_region:
            assert not any((b.layer[h] % 2 == 1 and b.layers[b.layer[h]]["kind"] == 0) for h in found)
            changed += int(r["n_hits"][t] != r_all["n_hits"][t])
        elif abs(np.arcsinh(1 / math.tan(b.true_state[5, b.seed_hits[0, t]]))) > 0.95:
            assert r["n_hits"][t] == r_all["n_hits"][t]
    assert changed > 10
