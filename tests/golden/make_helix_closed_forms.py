"""Writes helix_closed_forms.json: crossings of origin-centred cylinders by
tracks from the beam line, from textbook closed forms only (no oracle, no CUDA).

A particle of transverse momentum pT [GeV] in a field B [T] moves on a circle of
radius rho = pT / (0.0029979245800 B) cm (pT = 0.3 B R with R in metres).  From
the origin, the chord to radius R subtends the turning angle 2 a with
sin(a) = R / (2 rho); the transverse path is s = 2 rho a, the momentum turns by
2 a and the position azimuth by a (clockwise for positive charge in +Bz), and z
grows by s cot(theta).
"""
import json
import math
import os

K = 0.0029979245800
cases = []
for (pt, q, bz, R, phi0, theta, z0) in [
    (1.0, +1, 3.8, 50.0, 0.0, math.pi / 2, 0.0),
    (1.0, -1, 3.8, 50.0, 0.3, 1.0, 1.5),
    (0.6, +1, 3.8, 80.0, -2.0, 2.2, -3.0),
    (10.0, -1, 3.8, 100.0, 3.0, 0.5, 4.0),
    (2.0, +1, 2.0, 25.0, 1.0, 1.3, 0.0),
]:
    rho = pt / (K * bz)
    a = math.asin(R / (2 * rho))
    turn = -q
    s = 2 * rho * a
    pos = phi0 + turn * a
    cases.append(dict(pt=pt, q=q, bz=bz, R=R, phi0=phi0, theta=theta, z0=z0, s=s,
                      xyz=[R * math.cos(pos), R * math.sin(pos), z0 + s / math.tan(theta)],
                      phi=math.atan2(math.sin(phi0 + turn * 2 * a), math.cos(phi0 + turn * 2 * a)),
                      rho=rho))
out = dict(source="textbook helix closed forms (pT = 0.3 B R); see make_helix_closed_forms.py", cases=cases)
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "helix_closed_forms.json"), "w") as fh:
    json.dump(out, fh, indent=1)
