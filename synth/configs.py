"""Detector geometries and event configurations (synthetic stand-ins).

Units: cm, GeV, tesla, radians.  A layer is a barrel cylinder (kind 0, radius
`r_or_z`, z-extent [lo, hi]) or an endcap disk (kind 1, at z = `r_or_z`,
r-extent [lo, hi]), with a 2-D hit resolution: `sigma_u` along r-phi and
`sigma_v` along z (cylinder) or r (disk).  `n_phi` x `n_zr` is the hit-bin grid
the binning step uses for the layer (phi x z on cylinders, phi x r on disks).

The paper describes geometry as a vector of per-layer descriptions holding the
layer's dimensions, search-window parameters and flags (sec. 2.1); these tables
are that description for the three synthetic detectors used here.
"""
from __future__ import annotations

# Transverse momentum [GeV] = K_FIELD * B [T] * radius of curvature [cm].
K_FIELD = 0.0029979245800

UM = 1e-4  # one micrometre in cm


def _cyl(r, half, su, sv, nphi, nz):
    return dict(kind=0, r_or_z=float(r), lo=-float(half), hi=float(half),
                sigma_u=float(su), sigma_v=float(sv), n_phi=int(nphi), n_zr=int(nz))


def _disk(z, rlo, rhi, su, sv, nphi, nr):
    return dict(kind=1, r_or_z=float(z), lo=float(rlo), hi=float(rhi),
                sigma_u=float(su), sigma_v=float(sv), n_phi=int(nphi), n_zr=int(nr))


def _barrel10(nphi, nz):
    return [_cyl(4.0 + 96.0 * i / 9.0, 125.0, 20 * UM, 100 * UM, nphi, nz) for i in range(10)]


def _disks10(nphi, nr):
    out = []
    for sign in (+1.0, -1.0):
        for z in (120.0, 157.5, 195.0, 232.5, 270.0):
            out.append(_disk(sign * z, 4.0, 100.0, 20 * UM, 100 * UM, nphi, nr))
    return out


def _dense45(nphi, nz):
    lay = []
    for r in (3.0, 7.0, 11.0, 16.0):
        lay.append(_cyl(r, 27.0, 15 * UM, 15 * UM, nphi, nz))
    for i in range(13):
        lay.append(_cyl(25.0 + 85.0 * i / 12.0, 110.0, 30 * UM, 1000 * UM, nphi, nz))
    for sign in (+1.0, -1.0):
        for z in (32.0, 40.0, 50.0):
            lay.append(_disk(sign * z, 4.5, 16.0, 15 * UM, 15 * UM, nphi, nz))
        for i in range(11):
            lay.append(_disk(sign * (75.0 + 205.0 * i / 10.0), 20.0, 110.0, 30 * UM, 1000 * UM, nphi, nz))
    return lay


# Each config: geometry, field, track count and kinematic ranges, inefficiency,
# noise model.  pt_spectrum "flat" = uniform in [pt_min, pt_max]; "power3" =
# density proportional to pT^-3 on [pt_min, pt_max].
CONFIGS = {
    # KF fit only, 1 event x 1000 tracks, 10 barrel cylinders, |eta| < 1.
    "fit10": dict(layers=_barrel10(64, 8), bz=3.8, n_tracks=1000, eta_max=1.0,
                  pt_min=0.5, pt_max=10.0, pt_spectrum="flat", z0_half=5.0,
                  ineff=0.0, noise_mode="none", noise=0.0),
    # Same, without a field: straight lines.
    "fit10_b0": dict(layers=_barrel10(64, 8), bz=0.0, n_tracks=1000, eta_max=1.0,
                     pt_min=0.5, pt_max=10.0, pt_spectrum="flat", z0_half=5.0,
                     ineff=0.0, noise_mode="none", noise=0.0),
    # Track finding: 10 cylinders + 5 disks per side, |eta| < 2.4, 2 % inefficiency,
    # uniform noise at 5x each layer's signal count.
    "find20": dict(layers=_barrel10(256, 32) + _disks10(256, 32), bz=3.8, n_tracks=2000,
                   eta_max=2.4, pt_min=0.5, pt_max=10.0, pt_spectrum="flat", z0_half=5.0,
                   ineff=0.02, noise_mode="per_signal", noise=5.0),
    # Dense occupancy: 17 cylinders + 2 x 14 disks, pT^-3, 200k noise hits per event.
    "dense45": dict(layers=_dense45(256, 32), bz=3.8, n_tracks=6000, eta_max=2.4,
                    pt_min=0.5, pt_max=100.0, pt_spectrum="power3", z0_half=5.0,
                    ineff=0.02, noise_mode="total", noise=200000.0),
}

CONFIG_IDS = {name: i for i, name in enumerate(sorted(CONFIGS))}


def get_config(name: str) -> dict:
    if name not in CONFIGS:
        raise KeyError(f"unknown config {name!r}; known: {sorted(CONFIGS)}")
    return CONFIGS[name]


def layer_table(name_or_layers) -> list[dict]:
    """The layer list of a config (or a given list), as dictionaries."""
    if isinstance(name_or_layers, str):
        return [dict(d) for d in get_config(name_or_layers)["layers"]]
    return [dict(d) for d in name_or_layers]


def check_layers(layers) -> None:
    for i, d in enumerate(layers):
        if d["kind"] not in (0, 1):
            raise ValueError(f"layer {i}: kind must be 0 or 1")
        if not (d["hi"] > d["lo"]):
            raise ValueError(f"layer {i}: empty extent")
        if d["kind"] == 0 and not d["r_or_z"] > 0:
            raise ValueError(f"layer {i}: cylinder radius must be > 0")
        if d["kind"] == 1 and not (d["lo"] >= 0 and d["r_or_z"] != 0):
            raise ValueError(f"layer {i}: bad disk")
        if not (d["sigma_u"] > 0 and d["sigma_v"] > 0):
            raise ValueError(f"layer {i}: resolutions must be > 0")
