"""Seeded synthetic events: particles, layer crossings, smeared hits, noise, truth seeds.

Every random number comes from a counter-based Philox stream keyed by
(base seed 181104141, config id, event index), so an event is reproducible from
its three integers alone.

Particle motion (physics, not the fitting method): a particle of charge q and
transverse momentum pT in a uniform field Bz turns at the rate
h = -q * K_FIELD * Bz / pT per unit transverse path length s.  From the vertex
(0, 0, z0) with azimuth phi0 and polar angle theta,
    x(s) = (sin(phi0 + h s) - sin(phi0)) / h,  y(s) = -(cos(phi0 + h s) - cos(phi0)) / h,
    z(s) = z0 + s cot(theta),  with the straight line as the h = 0 case.
Hits are made only on the outward half-turn (0 < h s < pi), at most one per layer.
Cylinder crossings use the closed form from the beam line (the transverse
distance grows as |2 sin(h s / 2) / h|), which is a special case that neither
implementation of the method uses: both solve crossings from arbitrary points.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .configs import CONFIG_IDS, K_FIELD, get_config

BASE_SEED = 181104141
_S_MAX_STRAIGHT = 5000.0  # cm; path limit for a straight (B = 0) track


def _rng(config: str, event: int, base_seed: int = BASE_SEED) -> np.random.Generator:
    key = (int(base_seed) << 64) | (CONFIG_IDS[config] << 32) | (int(event) & 0xFFFFFFFF)
    return np.random.Generator(np.random.Philox(key=key))


def _helix_xy(h, phi0, s):
    """Transverse position after path s from the origin (vectorised, float64)."""
    h = np.asarray(h, dtype=np.float64)
    straight = h == 0.0
    hs = np.where(straight, 1.0, h)
    x = np.where(straight, s * np.cos(phi0), (np.sin(phi0 + h * s) - np.sin(phi0)) / hs)
    y = np.where(straight, s * np.sin(phi0), -(np.cos(phi0 + h * s) - np.cos(phi0)) / hs)
    return x, y


def _cylinder_crossings(h, phi0, radii, s_max):
    """Path length of each particle's outward crossing of each radius (NaN if none).

    From the beam line the transverse distance after path s is
    |2 sin(h s / 2) / h|, so the crossing of radius R is s = 2 asin(R |h| / 2) / |h|
    (s = R for a straight track), provided R <= 2 / |h|."""
    R = radii[None, :]
    ah = np.abs(h)[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        x = R * ah / 2.0
        s = np.where(ah == 0.0, R, 2.0 * np.arcsin(np.minimum(x, 1.0)) / np.where(ah == 0.0, 1.0, ah))
    s = np.where((ah == 0.0) | (x <= 1.0), s, np.nan)
    s = np.where(s < s_max[:, None], s, np.nan)
    # the crossing point must lie on the cylinder
    ok = ~np.isnan(s)
    if ok.any():
        hh = np.broadcast_to(h[:, None], s.shape)[ok]
        xx, yy = _helix_xy(hh, np.broadcast_to(phi0[:, None], s.shape)[ok], s[ok])
        assert np.allclose(np.hypot(xx, yy), np.broadcast_to(R, s.shape)[ok], rtol=1e-9, atol=1e-9)
    return s


PION_MASS = 0.13957  # GeV; mass hypothesis for the scattering angle


def _highland(p, x0_path):
    """RMS projected multiple-scattering angle (Highland, as tabulated by the
    Particle Data Group) for momentum p (GeV) through x0_path radiation lengths,
    unit charge, pion mass."""
    beta = p / np.sqrt(p * p + PION_MASS * PION_MASS)
    t = np.maximum(x0_path, 1e-12)
    return 0.0136 / (beta * p) * np.sqrt(t) * (1.0 + 0.038 * np.log(t / (beta * beta)))


def _cylinder_path_from(x, y, phi, h, R):
    """Transverse path from (x, y) with azimuth phi and turning rate h to the
    first crossing of radius R ahead (NaN if none): the intersection of the
    particle's circle (centre c, radius 1/|h|) with the circle of radius R; the
    straight line for h = 0."""
    with np.errstate(divide="ignore", invalid="ignore"):
        b = x * np.cos(phi) + y * np.sin(phi)
        disc = b * b - (x * x + y * y - R * R)
        s_line = np.where(disc >= 0, -b + np.sqrt(np.maximum(disc, 0.0)), np.nan)
        hs = np.where(h == 0.0, 1.0, h)
        cx, cy = x - np.sin(phi) / hs, y + np.cos(phi) / hs
        A, B = 2.0 * cx / hs, -2.0 * cy / hs
        M = np.hypot(A, B)
        qv = (R * R - cx * cx - cy * cy - 1.0 / (hs * hs)) / M
        a = np.arcsin(np.clip(qv, -1.0, 1.0))
        d = np.arctan2(B, A)
        best = np.full(np.shape(x), np.inf)
        for u in (a - d, np.pi - a - d):
            du = np.where(hs > 0, u - phi, phi - u)
            du = np.mod(du, 2.0 * np.pi)
            du = np.where(du <= 1e-12, 2.0 * np.pi, du)
            best = np.minimum(best, du / np.abs(hs))
        s_helix = np.where(np.abs(qv) <= 1.0, best, np.nan)
    return np.where(h == 0.0, s_line, s_helix)


def _scattered_cylinder_crossings(h, phi0, z0, theta, q, pt, bz, rz, lo, hi, x0, rng_ms, s_max, eloss=0.0):
    """Crossings of every cylinder (in radius order) with a multiple-scattering
    kick at each one crossed inside its z extent: the particle moves on a helix
    from crossing to crossing; at a crossing its polar angle and azimuth receive
    Gaussian kicks of width theta0 (Highland, path x0 / |cos| of the angle to
    the cylinder normal) and theta0 / sin(theta), the momentum magnitude staying
    the same (so q/pT follows theta); then, with eloss > 0 (GeV per radiation
    length at minimum ionisation), the particle loses the mean energy
    eloss * x / beta^2 for the same path x (no straggling).  x0 may also be an
    r-z material map (dict: r_max, z_min, z_max, x0 [nr, nz], eloss [nr, nz] or
    None; cells of equal size, points outside it in the nearest edge cell): each
    crossing then takes x0 and eloss from the cell holding its (r, z) and the
    eloss argument is not used.  Returns per (particle, layer) the path
    from the vertex, the crossing point, and (q/pT, phi, theta) after the kick;
    NaN where the cylinder is not reached."""
    P, L = h.shape[0], rz.shape[0]
    out = {k: np.full((P, L), np.nan) for k in ("S", "X", "Y", "Z", "W", "PHI", "TH")}
    x, y, z = np.zeros(P), np.zeros(P), z0.copy()
    phi, th = phi0.copy(), theta.copy()
    w = q / pt
    pmom = pt / np.sin(theta)
    s_tot, turned = np.zeros(P), np.zeros(P)
    alive = np.ones(P, dtype=bool)
    for l in np.argsort(rz):
        hh = -w * K_FIELD * bz
        s = _cylinder_path_from(x, y, phi, hh, rz[l])
        ok = alive & np.isfinite(s) & (turned + np.abs(hh) * np.nan_to_num(s) < np.pi) & (s_tot + np.nan_to_num(s) < s_max)
        sf = np.where(ok, s, 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            hsafe = np.where(hh == 0.0, 1.0, hh)
            xn = np.where(hh == 0.0, x + sf * np.cos(phi), x + (np.sin(phi + hh * sf) - np.sin(phi)) / hsafe)
            yn = np.where(hh == 0.0, y + sf * np.sin(phi), y - (np.cos(phi + hh * sf) - np.cos(phi)) / hsafe)
        zn = z + sf / np.tan(th)
        phin = phi + hh * sf
        inside = ok & (zn >= lo[l]) & (zn <= hi[l])
        if isinstance(x0, dict):
            nr, nz = np.shape(x0["x0"])
            ir = np.clip(np.floor(rz[l] / x0["r_max"] * nr), 0, nr - 1).astype(np.int64)
            iz = np.clip(np.floor((np.nan_to_num(zn) - x0["z_min"]) / (x0["z_max"] - x0["z_min"]) * nz),
                         0, nz - 1).astype(np.int64)
            x0v = np.asarray(x0["x0"], dtype=np.float64)[ir, iz]
            elv = (np.zeros(P) if x0.get("eloss") is None
                   else np.asarray(x0["eloss"], dtype=np.float64)[ir, iz])
        else:
            x0v, elv = np.full(P, float(x0)), np.full(P, float(eloss))
        # kick (drawn for every particle and layer, used where the layer is crossed)
        gk = rng_ms.standard_normal((P, 2))
        cosa = np.abs(np.sin(th) * np.cos(phin - np.arctan2(yn, xn)))
        t0 = np.where(x0v > 0.0, _highland(pmom, np.maximum(x0v, 1e-30) / np.maximum(cosa, 1e-6)), 0.0)
        th2 = np.where(inside, th + t0 * gk[:, 0], th)
        phi2 = np.where(inside, phin + t0 * gk[:, 1] / np.sin(th), phin)
        if (elv > 0.0).any():
            beta = pmom / np.sqrt(pmom * pmom + PION_MASS * PION_MASS)
            e_new = np.sqrt(pmom * pmom + PION_MASS * PION_MASS) - elv * (x0v / np.maximum(cosa, 1e-6)) / (beta * beta)
            stops = inside & (e_new <= PION_MASS)
            pmom = np.where(inside & ~stops, np.sqrt(np.maximum(e_new * e_new - PION_MASS * PION_MASS, 1e-30)), pmom)
            ok = ok & ~stops
        w2 = np.where(inside, np.sign(w) / (pmom * np.sin(th2)), w)
        sel = inside
        out["S"][sel, l] = (s_tot + sf)[sel]
        out["X"][sel, l], out["Y"][sel, l], out["Z"][sel, l] = xn[sel], yn[sel], zn[sel]
        out["W"][sel, l] = w2[sel]
        out["PHI"][sel, l] = np.arctan2(np.sin(phi2[sel]), np.cos(phi2[sel]))
        out["TH"][sel, l] = th2[sel]
        x, y, z = np.where(ok, xn, x), np.where(ok, yn, y), np.where(ok, zn, z)
        phi, th, w = np.where(ok, phi2, phi), np.where(ok, th2, th), np.where(ok, w2, w)
        turned = turned + np.where(ok, np.abs(hh) * sf, 0.0)
        s_tot = s_tot + sf
        alive = ok
    return out


def _scattered_crossings(h, phi0, z0, theta, q, pt, bz, kinds, rz, lo, hi, x0, rng_ms, s_max, eloss=0.0):
    """As _scattered_cylinder_crossings, for layouts with cylinders and disks:
    each particle moves on a helix from surface to surface, the next surface
    being the nearer in path of its next cylinder (by radius) and its next disk
    (by z in its direction of motion); a surface crossed inside its extent gets
    a hit, the Highland kick (path x0 / |cos| of the angle to the surface normal:
    sin(theta) cos(phi - phi_pos) on a cylinder, cos(theta) on a disk) and the
    mean energy loss; one that is crossed outside it is passed with no material.
    Normals are drawn for every particle at every step, in step order."""
    P, L = h.shape[0], rz.shape[0]
    out = {k: np.full((P, L), np.nan) for k in ("S", "X", "Y", "Z", "W", "PHI", "TH")}
    cyl = np.where(kinds == 0)[0]
    cyl = cyl[np.argsort(rz[cyl])]
    dsk = np.where(kinds == 1)[0]
    dsk = dsk[np.argsort(rz[dsk])]
    nc_, nd_ = cyl.size, dsk.size
    x, y, z = np.zeros(P), np.zeros(P), z0.copy()
    phi, th = phi0.copy(), theta.copy()
    w = q / pt
    pmom = pt / np.sin(theta)
    dirz = np.where(np.cos(theta) >= 0.0, 1, -1)
    # index of the first disk ahead of the vertex in each particle's direction
    if nd_:
        zd = rz[dsk]
        nd = np.where(dirz > 0, np.searchsorted(zd, z0, side="right"), np.searchsorted(zd, z0, side="left") - 1)
    else:
        nd = np.full(P, -1)
    nc = np.zeros(P, dtype=np.int64)
    s_tot, turned = np.zeros(P), np.zeros(P)
    alive = np.ones(P, dtype=bool)
    rows = np.arange(P)
    for _ in range(L + 1):
        if not alive.any():
            break
        hh = -w * K_FIELD * bz
        has_c = alive & (nc < nc_)
        Rc = np.where(has_c, rz[cyl[np.minimum(nc, max(nc_ - 1, 0))]] if nc_ else 0.0, 0.0)
        sc = np.where(has_c, _cylinder_path_from(x, y, phi, hh, np.where(has_c, Rc, 1.0)), np.nan)
        has_d = alive & (nd >= 0) & (nd < nd_)
        Zd = np.where(has_d, rz[dsk[np.clip(nd, 0, max(nd_ - 1, 0))]] if nd_ else 0.0, 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            sd = np.where(has_d, (Zd - z) * np.tan(th), np.nan)
        sd = np.where(sd > 0, sd, np.nan)
        use_c = np.isfinite(sc) & (~np.isfinite(sd) | (sc <= sd))
        s = np.where(use_c, sc, sd)
        ok = alive & np.isfinite(s) & (turned + np.abs(hh) * np.nan_to_num(s) < np.pi) & \
            (s_tot + np.nan_to_num(s) < s_max)
        l = np.where(use_c, cyl[np.minimum(nc, max(nc_ - 1, 0))] if nc_ else 0,
                     dsk[np.clip(nd, 0, max(nd_ - 1, 0))] if nd_ else 0)
        sf = np.where(ok, s, 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            hsafe = np.where(hh == 0.0, 1.0, hh)
            xn = np.where(hh == 0.0, x + sf * np.cos(phi), x + (np.sin(phi + hh * sf) - np.sin(phi)) / hsafe)
            yn = np.where(hh == 0.0, y + sf * np.sin(phi), y - (np.cos(phi + hh * sf) - np.cos(phi)) / hsafe)
        zn = np.where(use_c, z + sf / np.tan(th), Zd)
        phin = phi + hh * sf
        rn = np.hypot(xn, yn)
        inside = ok & np.where(use_c, (zn >= lo[l]) & (zn <= hi[l]), (rn >= lo[l]) & (rn <= hi[l]))
        x0v, elv = np.full(P, float(x0)), np.full(P, float(eloss))
        gk = rng_ms.standard_normal((P, 2))
        cosa = np.where(use_c, np.abs(np.sin(th) * np.cos(phin - np.arctan2(yn, xn))), np.abs(np.cos(th)))
        t0 = np.where(x0v > 0.0, _highland(pmom, np.maximum(x0v, 1e-30) / np.maximum(cosa, 1e-6)), 0.0)
        th2 = np.where(inside, th + t0 * gk[:, 0], th)
        phi2 = np.where(inside, phin + t0 * gk[:, 1] / np.sin(th), phin)
        if (elv > 0.0).any():
            beta = pmom / np.sqrt(pmom * pmom + PION_MASS * PION_MASS)
            e_new = np.sqrt(pmom * pmom + PION_MASS * PION_MASS) - elv * (x0v / np.maximum(cosa, 1e-6)) / (beta * beta)
            stops = inside & (e_new <= PION_MASS)
            pmom = np.where(inside & ~stops, np.sqrt(np.maximum(e_new * e_new - PION_MASS * PION_MASS, 1e-30)), pmom)
            ok = ok & ~stops
        w2 = np.where(inside, np.sign(w) / (pmom * np.sin(th2)), w)
        sel = inside
        li = l[sel]
        out["S"][rows[sel], li] = (s_tot + sf)[sel]
        out["X"][rows[sel], li], out["Y"][rows[sel], li], out["Z"][rows[sel], li] = xn[sel], yn[sel], zn[sel]
        out["W"][rows[sel], li] = w2[sel]
        out["PHI"][rows[sel], li] = np.arctan2(np.sin(phi2[sel]), np.cos(phi2[sel]))
        out["TH"][rows[sel], li] = th2[sel]
        x, y, z = np.where(ok, xn, x), np.where(ok, yn, y), np.where(ok, zn, z)
        phi, th, w = np.where(ok, phi2, phi), np.where(ok, th2, th), np.where(ok, w2, w)
        turned = turned + np.where(ok, np.abs(hh) * sf, 0.0)
        s_tot = s_tot + sf
        # the surface just reached is behind; a turned-back polar angle changes
        # the direction along z (the next disk is then the one behind)
        nc = np.where(ok & use_c, nc + 1, nc)
        nd = np.where(ok & ~use_c, nd + dirz, nd)
        nd_new_dir = np.where(np.cos(th) >= 0.0, 1, -1)
        flip = ok & (nd_new_dir != dirz)
        if flip.any() and nd_:
            nd = np.where(flip, np.where(nd_new_dir > 0, np.searchsorted(rz[dsk], z, side="right"),
                                          np.searchsorted(rz[dsk], z, side="left") - 1), nd)
            dirz = np.where(flip, nd_new_dir, dirz)
        alive = ok
    return out


def solenoid_field(bz, alpha, x, y, z):
    """Second-order solenoid field (tesla) at positions in cm: from the scalar
    potential solving Laplace's equation with axial symmetry,
    Bz = bz (1 - alpha (z^2 - r^2 / 2)), Bx = bz alpha x z, By = bz alpha y z."""
    return bz * alpha * x * z, bz * alpha * y * z, bz * (1.0 - alpha * (z * z - 0.5 * (x * x + y * y)))


def _field_rhs(bz, alpha, lam, r, t):
    """d(position)/dS, d(direction)/dS for unit charge with lam = q/p (1/GeV)."""
    bx, by, bzz = solenoid_field(bz, alpha, r[0], r[1], r[2])
    k = K_FIELD * lam
    dt = np.stack([k * (t[1] * bzz - t[2] * by), k * (t[2] * bx - t[0] * bzz), k * (t[0] * by - t[1] * bx)])
    return t, dt


def _field_step(bz, alpha, lam, r, t, d):
    """Classical Runge-Kutta step of path d (arrays of shape [3, n])."""
    a1, b1 = _field_rhs(bz, alpha, lam, r, t)
    a2, b2 = _field_rhs(bz, alpha, lam, r + 0.5 * d * a1, t + 0.5 * d * b1)
    a3, b3 = _field_rhs(bz, alpha, lam, r + 0.5 * d * a2, t + 0.5 * d * b2)
    a4, b4 = _field_rhs(bz, alpha, lam, r + d * a3, t + d * b3)
    return r + d / 6.0 * (a1 + 2 * a2 + 2 * a3 + a4), t + d / 6.0 * (b1 + 2 * b2 + 2 * b3 + b4)


FIELD_STEP = 0.5  # cm of path per generator step in the parameterised field


def _field_crossings(phi0, z0, theta, q, pt, bz, alpha, kinds, rz, lo, hi, ds=FIELD_STEP, s_max=2000.0):
    """Crossings of every layer by particles moving in the parameterised field
    (solenoid_field): the equation of motion integrated in fixed steps of ds cm
    of path from the vertex; a step that ends beyond a cylinder's radius (going
    out) or across a disk's plane is replaced, for that layer, by Newton steps
    from the step's start onto it.  A cylinder counts only on the way out (the
    first crossing), and nothing counts once the particle has turned by half a
    turn in the transverse plane or gone s_max cm (as with the helix: the
    outward half-turn), nor once it has left the volume of the layers (lo, hi:
    their extents).  Returns per (particle, layer) the path from the vertex,
    the crossing point and (q/pT, phi, theta) there (q/pT = q / (p sin theta)
    with |p| fixed); NaN where the layer is not crossed."""
    P, L = phi0.shape[0], rz.shape[0]
    out = {k: np.full((P, L), np.nan) for k in ("S", "X", "Y", "Z", "W", "PHI", "TH")}
    r = np.stack([np.zeros(P), np.zeros(P), z0.astype(np.float64)])
    t = np.stack([np.sin(theta) * np.cos(phi0), np.sin(theta) * np.sin(phi0), np.cos(theta)])
    lam = q * np.sin(theta) / pt
    S = np.zeros(P)
    turned = np.zeros(P)
    alive = np.ones(P, dtype=bool)
    done = np.zeros((P, L), dtype=bool)
    r_out = float(np.max(np.where(kinds == 0, rz, hi))) + 1.0
    z_out = float(np.max(np.where(kinds == 1, np.abs(rz), np.maximum(np.abs(lo), np.abs(hi))))) + 1.0
    cyl, dsk = np.nonzero(kinds == 0)[0], np.nonzero(kinds == 1)[0]
    while alive.any():
        idx = np.flatnonzero(alive)
        r0, t0 = r[:, idx], t[:, idx]
        rn, tn = _field_step(bz, alpha, lam[idx], r0, t0, ds)
        rho0, rhon = np.hypot(r0[0], r0[1]), np.hypot(rn[0], rn[1])
        for l in np.concatenate([cyl, dsk]):
            if kinds[l] == 0:
                hit = (rho0 < rz[l]) & (rhon >= rz[l]) & ~done[idx, l]
            else:
                hit = ((r0[2] - rz[l]) * (rn[2] - rz[l]) <= 0.0) & (r0[2] != rn[2]) & ~done[idx, l]
            if not hit.any():
                continue
            c = idx[hit]
            rc, tc, Sc = r0[:, hit], t0[:, hit], S[c].copy()
            for _n in range(6):
                if kinds[l] == 0:
                    rr = np.hypot(rc[0], rc[1])
                    d = (rz[l] - rr) / ((rc[0] * tc[0] + rc[1] * tc[1]) / rr)
                else:
                    d = (rz[l] - rc[2]) / tc[2]
                rc, tc = _field_step(bz, alpha, lam[c], rc, tc, d)
                Sc = Sc + d
            tt = np.hypot(tc[0], tc[1])
            th = np.arctan2(tt, tc[2])
            out["S"][c, l] = Sc
            out["X"][c, l], out["Y"][c, l], out["Z"][c, l] = rc[0], rc[1], rc[2]
            out["W"][c, l] = lam[c] / np.sin(th)
            out["PHI"][c, l] = np.arctan2(tc[1], tc[0])
            out["TH"][c, l] = th
            done[c, l] = True
        # transverse turning of the step (angle between the transverse directions)
        turned[idx] += np.abs(np.arctan2(t0[0] * tn[1] - t0[1] * tn[0], t0[0] * tn[0] + t0[1] * tn[1]))
        r[:, idx], t[:, idx] = rn, tn
        S[idx] += ds
        alive[idx] = (turned[idx] < np.pi) & (S[idx] < s_max) & (rhon < r_out) & (np.abs(rn[2]) < z_out)
    return out


@dataclass
class Batch:
    """A batch of events, hit arrays concatenated event after event.

    Hit arrays are indexed by the global hit index; `event_offsets[e]` is the first
    hit of event e.  Seeds are the first three hits (in path order) of every
    particle with at least three hits, in particle order.
    """
    config: str
    layers: list
    bz: float
    xyz: np.ndarray            # float32 [3, n_hits] SoA (the canonical input)
    xyz64: np.ndarray          # float64 [3, n_hits], values before rounding to float32
    layer: np.ndarray          # int32 [n_hits]
    hit_particle: np.ndarray   # int32 [n_hits], global particle id, -1 for noise
    event_offsets: np.ndarray  # int32 [n_events + 1]
    true_state: np.ndarray     # float64 [6, n_hits]: (x, y, z, q/pT, phi, theta) at the hit, NaN for noise
    true_xyz: np.ndarray       # float64 [3, n_hits]: unsmeared crossing point, NaN for noise
    seed_hits: np.ndarray      # int32 [3, n_seeds]
    seed_event: np.ndarray     # int32 [n_seeds]
    seed_particle: np.ndarray  # int32 [n_seeds]
    track_hits: np.ndarray     # int32 [max_hits, n_seeds], the particle's hits in path order, -1 padded
    particle_nhits: np.ndarray  # int32 [n_particles]
    particle_event: np.ndarray  # int32 [n_particles]
    particle_par: np.ndarray   # float64 [6, n_particles]: state at the vertex
    meta: dict = field(default_factory=dict)
    # seeds of overlap twins (make_batch(..., overlap=p)): for each seed, the index
    # of the seed it repeats with one hit replaced by that hit's twin, else -1
    seed_dup_of: np.ndarray = None

    @property
    def n_hits(self) -> int:
        return int(self.layer.shape[0])

    @property
    def n_events(self) -> int:
        return int(self.event_offsets.shape[0] - 1)

    @property
    def n_seeds(self) -> int:
        return int(self.seed_event.shape[0])

    def hit_bytes(self) -> int:
        return int(self.xyz.nbytes + self.layer.nbytes + self.event_offsets.nbytes)


def make_event(config: str, event: int, n_tracks: int | None = None, n_noise: int | None = None,
               base_seed: int = BASE_SEED, ineff: float | None = None, noise_scale: float = 1.0,
               eta_max: float | None = None, smear: bool = True, overlap: float = 0.0, material: float = 0.0,
               eloss: float = 0.0, field_alpha: float | None = None, material_map: dict | None = None):
    """One event as a dict of per-event arrays (local hit and particle indices).

    overlap > 0: each signal hit gets, with that probability, a second hit of the
    same particle on the same layer (overlapping sensors: the same crossing
    measured again with its own smearing).  These hits follow the noise hits and
    their random numbers are drawn after everything else, so the other arrays do
    not change.

    material > 0: every layer is that many radiation lengths thick at normal
    incidence and the particles scatter at each layer they cross (see
    _scattered_cylinder_crossings, and _scattered_crossings for layouts with
    disks); the kicks come from a stream of their own, so the other random
    numbers do not change.  eloss > 0 (with
    material): the mean energy loss per radiation length at minimum ionisation
    (GeV), lost at each layer crossed.

    field_alpha (no material): the particles move in the parameterised field
    solenoid_field(bz, field_alpha, ...) instead of the uniform one (see
    _field_crossings); no random numbers are drawn for it.

    material_map (layouts of cylinders only, instead of material / eloss): an
    r-z map (dict: r_max, z_min, z_max, x0 [nr, nz], eloss [nr, nz] or None)
    from which each crossing takes its material; the same random stream as
    material."""
    cfg = get_config(config)
    layers = cfg["layers"]
    rng = _rng(config, event, base_seed)
    P = int(cfg["n_tracks"] if n_tracks is None else n_tracks)
    eta_max = float(cfg["eta_max"] if eta_max is None else eta_max)
    ineff = float(cfg["ineff"] if ineff is None else ineff)
    bz = float(cfg["bz"])

    # Particle kinematics, drawn in a fixed order from the event's stream.
    u_pt = rng.random(P)
    if cfg["pt_spectrum"] == "flat":
        pt = cfg["pt_min"] + (cfg["pt_max"] - cfg["pt_min"]) * u_pt
    else:  # density ~ pT^-3 on [pt_min, pt_max], inverse CDF
        a, b = cfg["pt_min"] ** -2, cfg["pt_max"] ** -2
        pt = (a - u_pt * (a - b)) ** -0.5
    q = np.where(rng.random(P) < 0.5, -1.0, 1.0)
    phi0 = -np.pi + 2.0 * np.pi * rng.random(P)
    eta = -eta_max + 2.0 * eta_max * rng.random(P)
    z0 = -cfg["z0_half"] + 2.0 * cfg["z0_half"] * rng.random(P)
    theta = 2.0 * np.arctan(np.exp(-eta))
    cot = np.sinh(eta)
    h = -q * K_FIELD * bz / pt
    s_max = np.where(h == 0.0, _S_MAX_STRAIGHT, np.pi / np.where(h == 0.0, 1.0, np.abs(h)))

    kinds = np.array([d["kind"] for d in layers])
    rz = np.array([d["r_or_z"] for d in layers], dtype=np.float64)
    lo = np.array([d["lo"] for d in layers], dtype=np.float64)
    hi = np.array([d["hi"] for d in layers], dtype=np.float64)
    su = np.array([d["sigma_u"] for d in layers], dtype=np.float64)
    sv = np.array([d["sigma_v"] for d in layers], dtype=np.float64)
    L = len(layers)

    # Path length of each (particle, layer) crossing, NaN where there is none.
    S = np.full((P, L), np.nan)
    cyl = np.where(kinds == 0)[0]
    dsk = np.where(kinds == 1)[0]
    if cyl.size:
        S[:, cyl] = _cylinder_crossings(h, phi0, rz[cyl], s_max)
    if dsk.size:
        with np.errstate(divide="ignore", invalid="ignore"):
            sd = (rz[dsk][None, :] - z0[:, None]) / cot[:, None]
        ok = np.isfinite(sd) & (sd > 0) & (sd < s_max[:, None])
        S[:, dsk] = np.where(ok, sd, np.nan)
    ms = None
    if field_alpha is not None:
        if material > 0.0 or material_map is not None:
            raise ValueError("the parameterised field is supported without material")
        ms = _field_crossings(phi0, z0, theta, q, pt, bz, float(field_alpha), kinds, rz, lo, hi)
        S = ms["S"]
    elif material > 0.0 or material_map is not None:
        if material_map is not None and (material > 0.0 or eloss > 0.0):
            raise ValueError("give either material / eloss or material_map")
        if dsk.size and material_map is not None:
            raise ValueError("an r-z material map is supported for layouts of cylinders only")
        key = (int(base_seed) << 64) | (CONFIG_IDS[config] << 32) | (int(event) & 0xFFFFFFFF)
        rng_ms = np.random.Generator(np.random.Philox(key=key ^ (0x5CA77E8 << 96)))
        if dsk.size:
            ms = _scattered_crossings(h, phi0, z0, theta, q, pt, bz, kinds, rz, lo, hi, float(material), rng_ms,
                                      s_max, float(eloss))
        else:
            ms = _scattered_cylinder_crossings(h, phi0, z0, theta, q, pt, bz, rz, lo, hi,
                                               material_map if material_map is not None else float(material), rng_ms,
                                               s_max, float(eloss))
        S = ms["S"]
    Sf = np.where(np.isnan(S), 1.0, S)
    if ms is None:
        X, Y = _helix_xy(np.repeat(h[:, None], L, 1), np.repeat(phi0[:, None], L, 1), Sf)
        Z = z0[:, None] + Sf * cot[:, None]
    else:
        X, Y, Z = (np.where(np.isnan(ms[k]), 0.0, ms[k]) for k in ("X", "Y", "Z"))
    Rt = np.hypot(X, Y)
    in_ext = np.where(kinds[None, :] == 0, (Z >= lo[None, :]) & (Z <= hi[None, :]),
                      (Rt >= lo[None, :]) & (Rt <= hi[None, :]))
    crossed = ~np.isnan(S) & in_ext
    # Inefficiency: one uniform per (particle, layer), drawn for every pair.
    kept = crossed & (rng.random((P, L)) >= ineff)

    # Gaussian smearing: two normals per (particle, layer), drawn for every pair.
    g = rng.standard_normal((P, L, 2)) if smear else np.zeros((P, L, 2))
    phit = np.arctan2(Y, X)
    with np.errstate(divide="ignore", invalid="ignore"):
        ph_s = phit + g[:, :, 0] * su[None, :] / np.where(Rt > 0, Rt, 1.0)
    is_cyl = kinds[None, :] == 0
    r_s = np.where(is_cyl, rz[None, :], Rt + g[:, :, 1] * sv[None, :])
    z_s = np.where(is_cyl, Z + g[:, :, 1] * sv[None, :], rz[None, :])
    xs, ys = r_s * np.cos(ph_s), r_s * np.sin(ph_s)

    # Signal hits in particle order, then path order within a particle.
    flat = np.flatnonzero(kept)
    Sflat = S.ravel()[flat]
    order = np.lexsort((Sflat, flat // L))
    flat = flat[order]
    pid_l, lay_l = flat // L, flat % L
    ss = Sflat[order]
    n_sig = flat.size
    sig_xyz = np.empty((3, n_sig))
    sig_true_xyz = np.empty((3, n_sig))
    for k_, arr in enumerate((xs, ys, z_s)):
        sig_xyz[k_] = arr.ravel()[flat]
    for k_, arr in enumerate((X, Y, Z)):
        sig_true_xyz[k_] = arr.ravel()[flat]
    sig_state = np.empty((6, n_sig))
    sig_state[:3] = sig_true_xyz
    if ms is None:
        sig_state[3] = (q / pt)[pid_l]
        sig_state[4] = np.arctan2(np.sin(phi0[pid_l] + h[pid_l] * ss), np.cos(phi0[pid_l] + h[pid_l] * ss))
        sig_state[5] = theta[pid_l]
    else:  # after the layer's scattering
        sig_state[3] = ms["W"].ravel()[flat]
        sig_state[4] = ms["PHI"].ravel()[flat]
        sig_state[5] = ms["TH"].ravel()[flat]

    # Noise hits, uniform in (phi, z) on cylinders and uniform in area on disks.
    if cfg["noise_mode"] == "none" and n_noise is None:
        n_per_layer = np.zeros(L, dtype=np.int64)
    elif n_noise is not None or cfg["noise_mode"] == "total":
        tot = int(cfg["noise"] if n_noise is None else n_noise)
        tot = int(round(tot * noise_scale))
        n_per_layer = np.full(L, tot // L, dtype=np.int64)
        n_per_layer[0] += tot - int(n_per_layer.sum())
    else:
        n_sig = np.bincount(lay_l, minlength=L)
        n_per_layer = np.round(cfg["noise"] * noise_scale * n_sig).astype(np.int64)
    nz_layer = np.repeat(np.arange(L), n_per_layer)
    un = rng.random((nz_layer.size, 2))
    nph = -np.pi + 2.0 * np.pi * un[:, 0]
    k = kinds[nz_layer]
    nr = np.where(k == 0, rz[nz_layer], np.sqrt(lo[nz_layer] ** 2 + un[:, 1] * (hi[nz_layer] ** 2 - lo[nz_layer] ** 2)))
    nzc = np.where(k == 0, lo[nz_layer] + un[:, 1] * (hi[nz_layer] - lo[nz_layer]), rz[nz_layer])
    noise_xyz = np.stack([nr * np.cos(nph), nr * np.sin(nph), nzc])

    n_sig_hits = pid_l.size
    # Overlap twins: one uniform per signal hit, then two normals per twin.
    if overlap > 0.0:
        twin_of = np.flatnonzero(rng.random(n_sig_hits) < overlap)
        gt = rng.standard_normal((twin_of.size, 2)) if smear else np.zeros((twin_of.size, 2))
    else:
        twin_of = np.zeros(0, dtype=np.int64)
        gt = np.zeros((0, 2))
    tl = lay_l[twin_of]
    tx, ty, tz = sig_true_xyz[0, twin_of], sig_true_xyz[1, twin_of], sig_true_xyz[2, twin_of]
    trt = np.hypot(tx, ty)
    tcyl = kinds[tl] == 0
    with np.errstate(divide="ignore", invalid="ignore"):
        tph = np.arctan2(ty, tx) + gt[:, 0] * su[tl] / np.where(trt > 0, trt, 1.0)
    tr = np.where(tcyl, rz[tl], trt + gt[:, 1] * sv[tl])
    tzz = np.where(tcyl, tz + gt[:, 1] * sv[tl], rz[tl])
    twin_xyz = np.stack([tr * np.cos(tph), tr * np.sin(tph), tzz])

    xyz64 = np.concatenate([sig_xyz, noise_xyz, twin_xyz], axis=1)
    layer = np.concatenate([lay_l, nz_layer, tl]).astype(np.int32)
    particle = np.concatenate([pid_l, np.full(nz_layer.size, -1), pid_l[twin_of]]).astype(np.int32)
    true_state = np.concatenate([sig_state, np.full((6, nz_layer.size), np.nan), sig_state[:, twin_of]], axis=1)
    true_xyz = np.concatenate([sig_true_xyz, np.full((3, nz_layer.size), np.nan), sig_true_xyz[:, twin_of]], axis=1)
    nhits_p = np.bincount(pid_l, minlength=P).astype(np.int32)
    first = np.concatenate([[0], np.cumsum(nhits_p)[:-1]]).astype(np.int64)
    # local index of each twin, and of the signal hit it repeats
    twin_idx = n_sig_hits + nz_layer.size + np.arange(twin_of.size)
    return dict(xyz64=xyz64, layer=layer, particle=particle, true_state=true_state,
                true_xyz=true_xyz, nhits_p=nhits_p, first_hit_p=first, n_signal=n_sig_hits,
                twin_idx=twin_idx, twin_of=twin_of,
                par0=np.stack([np.zeros(P), np.zeros(P), z0, q / pt, phi0, theta]))


def _event_light(args):
    """make_event for a worker process, without the per-hit truth arrays and with
    the hit positions already rounded to float32 (what a timing run needs)."""
    config, ev, nt, nn, base_seed, kw = args
    p = make_event(config, ev, nt, nn, base_seed, **kw)
    p["xyz32"] = np.ascontiguousarray(p.pop("xyz64").astype(np.float32))
    for k in ("true_state", "true_xyz"):
        p.pop(k)
    return p


def make_batch(config: str, events, n_tracks=None, n_noise=None, base_seed: int = BASE_SEED,
               min_seed_hits: int = 3, workers: int = 1, truth: bool = True, **kw) -> Batch:
    """Concatenate events.  `n_tracks` / `n_noise` may be scalars or per-event lists.

    truth=False leaves out the per-hit truth arrays (true_state, true_xyz, xyz64
    are None); with workers > 1 (and truth=False) the events are generated in
    that many spawned processes.  The events are the same either way."""
    cfg = get_config(config)
    events = list(events)
    E = len(events)

    def per_event(v, i):
        if v is None or np.isscalar(v):
            return v
        return v[i]

    if truth:
        parts = [make_event(config, ev, per_event(n_tracks, i), per_event(n_noise, i), base_seed, **kw)
                 for i, ev in enumerate(events)]
    else:
        jobs = [(config, ev, per_event(n_tracks, i), per_event(n_noise, i), base_seed, kw)
                for i, ev in enumerate(events)]
        if workers > 1 and E > 1:
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            with ProcessPoolExecutor(max_workers=min(workers, E), mp_context=mp.get_context("spawn")) as ex:
                parts = list(ex.map(_event_light, jobs, chunksize=max(1, E // (4 * workers))))
        else:
            parts = [_event_light(j) for j in jobs]
    max_hits = max([1] + [int(p["nhits_p"].max(initial=0)) for p in parts])
    offs = np.zeros(E + 1, dtype=np.int64)
    xyz64, layer, hp, ts, tx = [], [], [], [], []
    seed_hits, seed_event, seed_part, track_hits, seed_dup = [], [], [], [], []
    p_nh, p_ev, p_par = [], [], []
    pbase = 0
    for i, p in enumerate(parts):
        base = offs[i]
        n = p["layer"].shape[0]
        offs[i + 1] = base + n
        xyz64.append(p["xyz64"] if truth else p["xyz32"]); layer.append(p["layer"])
        if truth:
            ts.append(p["true_state"]); tx.append(p["true_xyz"])
        hp.append(np.where(p["particle"] >= 0, p["particle"] + pbase, -1).astype(np.int32))
        P = p["nhits_p"].shape[0]
        ok = np.nonzero(p["nhits_p"] >= min_seed_hits)[0]
        f = p["first_hit_p"][ok]
        sh = np.stack([f, f + 1, f + 2])
        th = np.full((max_hits, ok.size), -1, dtype=np.int64)
        for j in range(max_hits):
            valid = j < p["nhits_p"][ok]
            th[j, valid] = f[valid] + j
        dup = np.full(ok.size, -1, dtype=np.int64)
        # a twin of a seed hit gives the particle a second seed (that hit replaced)
        if p["twin_of"].size:
            first_of = np.full(p["n_signal"], -1, dtype=np.int64)  # seed index of each signal hit in a seed
            slot_of = np.full(p["n_signal"], -1, dtype=np.int64)
            for k in range(3):
                first_of[sh[k]] = np.arange(ok.size)
                slot_of[sh[k]] = k
            sel = first_of[p["twin_of"]] >= 0
            ds, dk, dt = first_of[p["twin_of"][sel]], slot_of[p["twin_of"][sel]], p["twin_idx"][sel]
            sh2, th2 = sh[:, ds].copy(), th[:, ds].copy()
            sh2[dk, np.arange(ds.size)] = dt
            th2[dk, np.arange(ds.size)] = dt
            sh, th = np.concatenate([sh, sh2], axis=1), np.concatenate([th, th2], axis=1)
            dup = np.concatenate([dup, ds + sum(x.shape[1] for x in seed_hits)])
            ok = np.concatenate([ok, ok[ds]])
        seed_hits.append(sh + base)
        seed_event.append(np.full(ok.size, i))
        seed_part.append(ok + pbase)
        track_hits.append(np.where(th >= 0, th + base, -1))
        seed_dup.append(dup)
        p_nh.append(p["nhits_p"]); p_ev.append(np.full(P, i)); p_par.append(p["par0"])
        pbase += P
    if offs[-1] >= (1 << 28) - 2:
        raise ValueError("too many hits for 28-bit hit indices")
    xyz64 = np.concatenate(xyz64, axis=1)
    xyz32 = np.ascontiguousarray(xyz64.astype(np.float32)) if truth else xyz64
    if not truth:
        xyz64 = None
    layers = [dict(d) for d in cfg["layers"]]
    if kw.get("material", 0.0) > 0.0:
        for d in layers:
            d["x0"] = float(kw["material"])
            if kw.get("eloss", 0.0) > 0.0:
                d["eloss"] = float(kw["eloss"])
    return Batch(
        config=config, layers=layers, bz=float(cfg["bz"]),
        xyz=xyz32, xyz64=xyz64,
        layer=np.concatenate(layer).astype(np.int32), hit_particle=np.concatenate(hp).astype(np.int32),
        event_offsets=offs.astype(np.int32), true_state=np.concatenate(ts, axis=1) if truth else None,
        true_xyz=np.concatenate(tx, axis=1) if truth else None,
        seed_hits=np.ascontiguousarray(np.concatenate(seed_hits, axis=1).astype(np.int32)),
        seed_event=np.concatenate(seed_event).astype(np.int32),
        seed_particle=np.concatenate(seed_part).astype(np.int32),
        track_hits=np.ascontiguousarray(np.concatenate(track_hits, axis=1).astype(np.int32)),
        particle_nhits=np.concatenate(p_nh).astype(np.int32),
        particle_event=np.concatenate(p_ev).astype(np.int32),
        particle_par=np.concatenate(p_par, axis=1),
        meta=dict(events=events, base_seed=base_seed, field_alpha=kw.get("field_alpha"),
              material_map=kw.get("material_map")),
        seed_dup_of=np.concatenate(seed_dup).astype(np.int32),
    )
