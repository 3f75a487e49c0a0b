"""FP64 CPU oracle for the Kalman-filter fit and find (test infrastructure only).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The product path (the CUDA library and its binding)
never does.  The arithmetic lives in `mkf_oracle.c` (plain C, double precision);
this module compiles it with gcc on first use and marshals numpy arrays.

Parity status of each function is stated in the oracle's test modules
(tests/test_oracle_pins.py and, for the field, material map, smoother, seed
cleaning, MLP and learned pruning, the other tests/test_oracle_*.py); every
exported function here is pinned there.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mkf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_UNREACHABLE = 1
ST_BADSEED = 2
ST_NONFINITE = 4
ST_BADS = 8
ST_MISSSTOP = 16
ST_TRUNC = 32


def build(force: bool = False) -> str:
    """Compile the oracle into liboracle.so (plain gcc, -O2, no OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            d, i32, i64, u64 = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_uint64)
            u32 = C.POINTER(C.c_uint32)
            geom = [C.c_int, i32, d, d, d, d, d, d, d, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int,
                    C.c_double, C.c_double, C.c_double, d, d, C.c_int, d, u64]
            lib.or_field.argtypes = geom + [d, d]
            lib.or_field.restype = C.c_int
            lib.or_propagate.argtypes = geom + [d, C.c_int, d, d, d]
            lib.or_propagate.restype = C.c_int
            lib.or_helix_move.argtypes = geom + [d, C.c_double, d]
            lib.or_helix_move.restype = C.c_int
            lib.or_transport.argtypes = [d, d, d]
            lib.or_transport.restype = None
            lib.or_update.argtypes = geom + [C.c_int, d, d, d, d, d, d]
            lib.or_update.restype = C.c_double
            lib.or_seed.argtypes = geom + [d, d, d, C.c_int, d, d]
            lib.or_seed.restype = C.c_int
            lib.or_scattering.argtypes = geom + [C.c_int, d, d]
            lib.or_scattering.restype = C.c_int
            lib.or_eloss.argtypes = geom + [C.c_int, d, d, C.c_double]
            lib.or_eloss.restype = C.c_int
            lib.or_fit.argtypes = geom + [d, C.c_int64, i32, i32, C.c_int, C.c_int64, d, d, d, d, d, i32, u32]
            lib.or_fit.restype = C.c_int
            lib.or_fit_backward.argtypes = geom + [d, C.c_int64, i32, i32, C.c_int, C.c_int64, d, d, C.c_double, d, d,
                                                   d, i32, u32]
            lib.or_fit_backward.restype = C.c_int
            lib.or_fit_smooth.argtypes = geom + [d, C.c_int64, i32, i32, C.c_int, C.c_int64, d, d, C.c_double, d, d,
                                                 d, i32, u32, d]
            lib.or_fit_smooth.restype = C.c_int
            lib.or_find.argtypes = geom + [d, C.c_int64, i32, i32, C.c_int, i32, i32, C.c_int64, i64, C.c_int64,
                                           C.c_int, C.c_double, C.c_int, d, d, d, i32, i32, C.c_int, u32, i64, d,
                                           d, C.c_double, d, i32, i64, C.c_int64]
            lib.or_find.restype = C.c_int
            lib.or_mlp_logit.argtypes = [d, d, C.c_int64, d]
            lib.or_mlp_logit.restype = None
            _lib = lib
    return _lib


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


class Geometry:
    """Layer table + field + optional tracking regions (layer masks by seed eta)."""

    def __init__(self, layers, bz, region_edges=None, region_masks=None, field_alpha=None, material_map=None):
        self.layers = [dict(d) for d in layers]
        self.n = len(layers)
        self.kind = np.ascontiguousarray([d["kind"] for d in layers], dtype=np.int32)
        self.rz = np.ascontiguousarray([d["r_or_z"] for d in layers], dtype=np.float64)
        self.lo = np.ascontiguousarray([d["lo"] for d in layers], dtype=np.float64)
        self.hi = np.ascontiguousarray([d["hi"] for d in layers], dtype=np.float64)
        self.su = np.ascontiguousarray([d["sigma_u"] for d in layers], dtype=np.float64)
        self.sv = np.ascontiguousarray([d["sigma_v"] for d in layers], dtype=np.float64)
        # material: radiation lengths at normal incidence (optional "x0" key)
        self.x0 = np.ascontiguousarray([d.get("x0", 0.0) for d in layers], dtype=np.float64)
        # mean energy loss per radiation length at minimum ionisation, GeV (optional "eloss")
        self.eloss = np.ascontiguousarray([d.get("eloss", 0.0) for d in layers], dtype=np.float64)
        self.bz = float(bz)
        # field: uniform (None) or parameterised with fall-off coefficient alpha
        # (1/cm^2; alpha = 0 is the uniform field integrated numerically)
        self.field_kind = 0 if field_alpha is None else 1
        self.alpha = 0.0 if field_alpha is None else float(field_alpha)
        # r-z material map: dict(r_max, z_min, z_max, x0 [nr, nz], eloss [nr, nz] or
        # None); it replaces the layers' own material values
        self.material_map = material_map
        if material_map is None:
            self.map_args = [0, 0, 0.0, 0.0, 0.0, None, None]
        else:
            mx = np.ascontiguousarray(material_map["x0"], dtype=np.float64)
            me = material_map.get("eloss")
            me = None if me is None else np.ascontiguousarray(me, dtype=np.float64)
            self._map = (mx, me)
            self.map_args = [mx.shape[0], mx.shape[1], float(material_map["r_max"]), float(material_map["z_min"]),
                             float(material_map["z_max"]), _p(mx, C.c_double), _p(me, C.c_double)]
        edges = [] if region_edges is None else list(region_edges)
        self.n_regions = len(edges) + 1
        self.edges = np.ascontiguousarray(edges + [0.0], dtype=np.float64)
        if region_masks is None:
            region_masks = [(1 << self.n) - 1] * self.n_regions
        self.masks = np.ascontiguousarray(region_masks, dtype=np.uint64)

    def args(self):
        return [self.n, _p(self.kind, C.c_int32), _p(self.rz, C.c_double), _p(self.lo, C.c_double),
                _p(self.hi, C.c_double), _p(self.su, C.c_double), _p(self.sv, C.c_double),
                _p(self.x0, C.c_double), _p(self.eloss, C.c_double), self.bz, self.field_kind, self.alpha,
                *self.map_args, self.n_regions,
                _p(self.edges, C.c_double),
                _p(self.masks, C.c_uint64)]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def propagate(geo: Geometry, p, layer):
    """Propagate state p to `layer`: (q, J (6x6), s) or None if unreachable."""
    lib = _load()
    p = _f64(p)
    q, J, s = np.zeros(6), np.zeros(36), np.zeros(1)
    rc = lib.or_propagate(*geo.args(), _p(p, C.c_double), int(layer), _p(q, C.c_double), _p(J, C.c_double),
                          _p(s, C.c_double))
    if rc < 0:
        raise ValueError("bad arguments")
    if rc == 0:
        return None
    return q, J.reshape(6, 6), float(s[0])


def helix_move(geo: Geometry, p, s):
    lib = _load()
    p = _f64(p)
    q = np.zeros(6)
    lib.or_helix_move(*geo.args(), _p(p, C.c_double), float(s), _p(q, C.c_double))
    return q


def transport(J, Cm):
    lib = _load()
    J, Cm = _f64(J).reshape(36), _f64(Cm).reshape(36)
    out = np.zeros(36)
    lib.or_transport(_p(J, C.c_double), _p(Cm, C.c_double), _p(out, C.c_double))
    return out.reshape(6, 6)


def update(geo: Geometry, layer, hit, p, Cm):
    """Kalman update: returns (p', C', chi2, r, S, C_joseph)."""
    lib = _load()
    p, Cm, hit = _f64(p).copy(), _f64(Cm).reshape(36).copy(), _f64(hit)
    r, S, Cj = np.zeros(2), np.zeros(4), np.zeros(36)
    chi2 = lib.or_update(*geo.args(), int(layer), _p(hit, C.c_double), _p(p, C.c_double), _p(Cm, C.c_double),
                         _p(r, C.c_double), _p(S, C.c_double), _p(Cj, C.c_double))
    return p, Cm.reshape(6, 6), float(chi2), r, S.reshape(2, 2), Cj.reshape(6, 6)


def scattering(geo: Geometry, layer, p):
    """Multiple-scattering noise (6x6) the material of `layer` adds at state p."""
    lib = _load()
    p = _f64(p)
    Q = np.zeros(36)
    if lib.or_scattering(*geo.args(), int(layer), _p(p, C.c_double), _p(Q, C.c_double)) < 0:
        raise ValueError("bad arguments")
    return Q.reshape(6, 6)


def eloss(geo: Geometry, layer, p, Cm, sign=1.0):
    """Mean energy loss (sign +1) or gain (-1) where p crosses `layer`:
    (p', C') from the state p and covariance Cm (6x6)."""
    lib = _load()
    p = _f64(p).copy()
    Cm = _f64(Cm).reshape(36).copy()
    if lib.or_eloss(*geo.args(), int(layer), _p(p, C.c_double), _p(Cm, C.c_double), float(sign)) < 0:
        raise ValueError("bad arguments")
    return p, Cm.reshape(6, 6)


def seed(geo: Geometry, h1, h2, h3, layer1):
    lib = _load()
    p, Cm = np.zeros(6), np.zeros(36)
    ok = lib.or_seed(*geo.args(), _p(_f64(h1), C.c_double), _p(_f64(h2), C.c_double), _p(_f64(h3), C.c_double),
                     int(layer1), _p(p, C.c_double), _p(Cm, C.c_double))
    return (p, Cm.reshape(6, 6)) if ok == 1 else None


def unpack21(c21):
    """[21, n] packed lower triangle -> [n, 6, 6]."""
    c21 = np.asarray(c21)
    n = c21.shape[1]
    out = np.zeros((n, 6, 6), dtype=c21.dtype)
    k = 0
    for i in range(6):
        for j in range(i + 1):
            out[:, i, j] = c21[k]
            out[:, j, i] = c21[k]
            k += 1
    return out


def pack21(Cm):
    """[n, 6, 6] -> [21, n]."""
    Cm = np.asarray(Cm)
    return np.stack([Cm[:, i, j] for i in range(6) for j in range(i + 1)])


def fit(geo: Geometry, xyz, hit_layer, hit_idx, seed_par=None, seed_cov21=None):
    """Kalman fit along fixed hit lists.  xyz [3, n_hits]; hit_idx [max_hits, n]."""
    lib = _load()
    xyz = _f64(xyz)
    n_hits = xyz.shape[1]
    hit_layer = np.ascontiguousarray(hit_layer, dtype=np.int32)
    hit_idx = np.ascontiguousarray(hit_idx, dtype=np.int32)
    max_hits, n = hit_idx.shape
    par, cov = np.zeros((6, n)), np.zeros((21, n))
    chi2, ndf, st = np.zeros(n), np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.uint32)
    sp = None if seed_par is None else _f64(seed_par)
    sc = None if seed_cov21 is None else _f64(seed_cov21)
    rc = lib.or_fit(*geo.args(), _p(xyz, C.c_double), n_hits, _p(hit_layer, C.c_int32), _p(hit_idx, C.c_int32),
                    max_hits, n, _p(sp, C.c_double), _p(sc, C.c_double), _p(par, C.c_double), _p(cov, C.c_double),
                    _p(chi2, C.c_double), _p(ndf, C.c_int32), _p(st, C.c_uint32))
    if rc != 0:
        raise RuntimeError(f"or_fit failed: {rc}")
    return dict(par=par, cov=cov, chi2=chi2, ndf=ndf, status=st)


def fit_backward(geo: Geometry, xyz, hit_layer, hit_idx, last_par, last_cov21, inflate=100.0):
    """Backward fit along fixed hit lists (hits in path order) from the state at
    each track's last hit (last_par [6, n], last_cov21 [21, n]); returns the state
    at the first hit with chi2 and ndf over every hit used."""
    lib = _load()
    xyz = _f64(xyz)
    n_hits = xyz.shape[1]
    hit_layer = np.ascontiguousarray(hit_layer, dtype=np.int32)
    hit_idx = np.ascontiguousarray(hit_idx, dtype=np.int32)
    max_hits, n = hit_idx.shape
    par, cov = np.zeros((6, n)), np.zeros((21, n))
    chi2, ndf, st = np.zeros(n), np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.uint32)
    lp, lc = _f64(last_par), _f64(last_cov21)
    rc = lib.or_fit_backward(*geo.args(), _p(xyz, C.c_double), n_hits, _p(hit_layer, C.c_int32),
                             _p(hit_idx, C.c_int32), max_hits, n, _p(lp, C.c_double), _p(lc, C.c_double),
                             C.c_double(inflate), _p(par, C.c_double), _p(cov, C.c_double), _p(chi2, C.c_double),
                             _p(ndf, C.c_int32), _p(st, C.c_uint32))
    if rc != 0:
        raise RuntimeError(f"or_fit_backward failed: {rc}")
    return dict(par=par, cov=cov, chi2=chi2, ndf=ndf, status=st)


def fit_smooth(geo: Geometry, xyz, hit_layer, hit_idx, seed_par=None, seed_cov21=None, inflate=100.0):
    """Smoothed state at every hit of fixed hit lists (two filters): par
    [max_hits, 6, n], cov [max_hits, 21, n] per row of hit_idx (NaN where none),
    the forward fit's chi2, ndf, status, and per track `shrink`, the largest
    ratio of a predicted residual variance to the hit's variance met by the
    backward filter (an update there shrinks its prior by about that factor)."""
    lib = _load()
    xyz = _f64(xyz)
    hl = np.ascontiguousarray(hit_layer, dtype=np.int32)
    hi = np.ascontiguousarray(hit_idx, dtype=np.int32)
    mh, n = hi.shape
    par, cov = np.zeros((mh, 6, n)), np.zeros((mh, 21, n))
    chi2, ndf, st, shrink = np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.uint32), np.zeros(n)
    sp = None if seed_par is None else _f64(seed_par)
    sc = None if seed_cov21 is None else _f64(seed_cov21)
    rc = lib.or_fit_smooth(*geo.args(), _p(xyz, C.c_double), xyz.shape[1], _p(hl, C.c_int32), _p(hi, C.c_int32), mh,
                           n, _p(sp, C.c_double), _p(sc, C.c_double), float(inflate), _p(par, C.c_double),
                           _p(cov, C.c_double), _p(chi2, C.c_double), _p(ndf, C.c_int32), _p(st, C.c_uint32),
                           _p(shrink, C.c_double))
    if rc < 0:
        raise ValueError("bad arguments")
    return dict(par=par, cov=cov, chi2=chi2, ndf=ndf, status=st, shrink=shrink)


def find(geo: Geometry, xyz, hit_layer, event_offsets, seed_hits, seed_event, n_best=10, chi2_cut=30.0,
         max_consec=3, seed_list=None, max_out=None, mlp_w=None, mlp_tau=0.0, dump_cap=0):
    """Track finding (n_best = 1: best hit; > 1: N best candidates per seed).
    mlp_w: 897 MLP weights (use the bfloat16-rounded values) turns on pruning at
    mlp_tau; dump_cap > 0 returns the features of compatible hits."""
    lib = _load()
    xyz = _f64(xyz)
    n_hits = xyz.shape[1]
    hit_layer = np.ascontiguousarray(hit_layer, dtype=np.int32)
    event_offsets = np.ascontiguousarray(event_offsets, dtype=np.int32)
    seed_hits = np.ascontiguousarray(seed_hits, dtype=np.int32)
    seed_event = np.ascontiguousarray(seed_event, dtype=np.int32)
    n_seeds = seed_hits.shape[1]
    sl = None if seed_list is None else np.ascontiguousarray(seed_list, dtype=np.int64)
    nl = n_seeds if sl is None else sl.shape[0]
    if max_out is None:
        max_out = geo.n + 3
    par, cov = np.zeros((6, nl)), np.zeros((21, nl))
    chi2, nh = np.zeros(nl), np.zeros(nl, dtype=np.int32)
    hits = np.zeros((max_out, nl), dtype=np.int32)
    st = np.zeros(nl, dtype=np.uint32)
    cnt = np.zeros((3, nl), dtype=np.int64)
    marg = np.zeros((4, nl))
    mw = None if mlp_w is None else _f64(mlp_w)
    feat = np.zeros((max(1, dump_cap), 12)) if dump_cap else None
    fref = np.zeros((max(1, dump_cap), 3), dtype=np.int32) if dump_cap else None
    fcnt = np.zeros(1, dtype=np.int64)
    rc = lib.or_find(*geo.args(), _p(xyz, C.c_double), n_hits, _p(hit_layer, C.c_int32),
                     _p(event_offsets, C.c_int32), event_offsets.shape[0] - 1, _p(seed_hits, C.c_int32),
                     _p(seed_event, C.c_int32), n_seeds, _p(sl, C.c_int64), nl, int(n_best), float(chi2_cut),
                     int(max_consec), _p(par, C.c_double), _p(cov, C.c_double), _p(chi2, C.c_double),
                     _p(nh, C.c_int32), _p(hits, C.c_int32), int(max_out), _p(st, C.c_uint32), _p(cnt, C.c_int64),
                     _p(marg, C.c_double), _p(mw, C.c_double), float(mlp_tau), _p(feat, C.c_double),
                     _p(fref, C.c_int32), _p(fcnt, C.c_int64), int(dump_cap))
    if rc != 0:
        raise RuntimeError(f"or_find failed: {rc}")
    out = dict(par=par, cov=cov, chi2=chi2, n_hits=nh, hits=hits, status=st, counters=cnt, margins=marg)
    if dump_cap:
        k = int(min(fcnt[0], dump_cap))
        out.update(feat=feat[:k], feat_ref=fref[:k], feat_count=int(fcnt[0]))
    return out


def mlp_logit(w, feat):
    """The finder's MLP score of feature rows feat [n, 12] with weights w [897]
    (as or_find applies it when pruning)."""
    lib = _load()
    w = _f64(w)
    feat = _f64(feat).reshape(-1, 12)
    out = np.zeros(feat.shape[0])
    lib.or_mlp_logit(_p(w, C.c_double), _p(feat, C.c_double), feat.shape[0], _p(out, C.c_double))
    return out


def geometry_for(batch, region_edges=None, region_masks=None) -> Geometry:
    """The batch's geometry with its values as the generator defines them
    (e.g. cylinder radii 4 + 96 i / 9 cm exactly)."""
    return Geometry(batch.layers, batch.bz, region_edges, region_masks, batch.meta.get("field_alpha"),
                    batch.meta.get("material_map"))


def _f32(v):
    return float(np.float32(v))


def geometry_as_loaded(batch, region_edges=None, region_masks=None, field_alpha="batch") -> Geometry:
    """The batch's geometry with every real-valued entry rounded to FP32, the
    precision in which the library's geometry calls take it (layer radii and
    z positions, extents, resolutions, material, field strength and fall-off,
    region edges, material-map cells and bounds).  A comparison of the library
    with the oracle gives both the same problem: the radius of a cylinder at
    4 + 96 i / 9 cm moves by up to 1.9e-6 cm when rounded to FP32, which shifts
    the crossing point of a track and its residuals by about 1e-3 of a 20 um
    resolution.  field_alpha: the batch's own field unless given (None = uniform)."""
    layers = []
    for d in batch.layers:
        e = dict(d)
        for k in ("r_or_z", "lo", "hi", "sigma_u", "sigma_v", "x0", "eloss"):
            if k in e:
                e[k] = _f32(e[k])
        layers.append(e)
    alpha = batch.meta.get("field_alpha") if isinstance(field_alpha, str) else field_alpha
    mm = batch.meta.get("material_map")
    if mm is not None:
        mm = dict(mm)
        for k in ("r_max", "z_min", "z_max"):
            mm[k] = _f32(mm[k])
        mm["x0"] = np.asarray(mm["x0"], dtype=np.float32).astype(np.float64)
        if mm.get("eloss") is not None:
            mm["eloss"] = np.asarray(mm["eloss"], dtype=np.float32).astype(np.float64)
    edges = None if region_edges is None else [_f32(x) for x in region_edges]
    return Geometry(layers, _f32(batch.bz), edges, region_masks, None if alpha is None else _f32(alpha), mm)


def field(geo: Geometry, r):
    """The field (T) at position r (cm)."""
    lib = _load()
    r = _f64(r)
    B = np.zeros(3)
    if lib.or_field(*geo.args(), _p(r, C.c_double), _p(B, C.c_double)) < 0:
        raise ValueError("bad arguments")
    return B
