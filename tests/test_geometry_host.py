"""CPU checks of the library's geometry-table construction (the host code behind
mkf_geometry_load), compiled for the host: validation errors, the radius- and
z-sorted layer lists, the per-layer bin layout, the z-extent bounds used by the
next-layer shortcut, and the tracking-region masks."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1811_04141_gb300 import _native as N
from synth import configs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1811_04141_gb300", "csrc")
MKF_OK, ERR_ARG, ERR_GEOMETRY, ERR_CAPACITY = 0, -1, -2, -3


@pytest.fixture(scope="module")
def lib():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "geom.so")
    subprocess.run([gxx, "-O1", "-std=c++17", "-fPIC", "-shared", "-I" + CSRC, "-I" + os.path.join(ROOT, "include"),
                    "-o", so, os.path.join(HERE, "host", "geom_host.cpp")], check=True)
    return C.CDLL(so)


def _layers(ls):
    arr = (N.MkfLayer * max(1, len(ls)))()
    for i, d in enumerate(ls):
        arr[i] = N.MkfLayer(int(d["kind"]), float(d["r_or_z"]), float(d["lo"]), float(d["hi"]), float(d["sigma_u"]),
                            float(d["sigma_v"]), int(d["n_phi"]), int(d["n_zr"]))
    return arr


def build(lib, ls, plans=None, edges=None, bz=3.8):
    out = np.zeros(256, np.int32)
    outf = np.zeros(160, np.float32)
    keep = []
    parr = None
    np_ = 0 if plans is None else len(plans)
    if np_:
        parr = (N.MkfPlan * np_)()
        for r, ids in enumerate(plans):
            a = (C.c_int32 * max(1, len(ids)))(*ids)
            keep.append(a)
            parr[r] = N.MkfPlan(len(ids), C.cast(a, C.POINTER(C.c_int32)))
    e = None if edges is None else (C.c_float * max(1, len(edges)))(*edges)
    st = lib.host_build_geom(_layers(ls), len(ls), parr, np_, e, C.c_float(bz), out.ctypes.data_as(C.c_void_p),
                             outf.ctypes.data_as(C.c_void_p))
    return st, out, outf


def test_dense_geometry_tables(lib):
    ls = configs.layer_table("dense45")
    st, out, outf = build(lib, ls)
    assert st == MKF_OK
    kinds = np.array([d["kind"] for d in ls])
    rz = np.array([d["r_or_z"] for d in ls])
    n_cyl, n_dsk = int((kinds == 0).sum()), int((kinds == 1).sum())
    assert out[0] == n_cyl and out[1] == n_dsk
    sizes = np.array([d["n_phi"] * d["n_zr"] for d in ls])
    assert out[2] == sizes.sum()
    assert np.array_equal(out[3:3 + len(ls)], np.concatenate([[0], np.cumsum(sizes)[:-1]]))
    cyl = out[67:67 + n_cyl]
    dsk = out[131:131 + n_dsk]
    assert (kinds[cyl] == 0).all() and (np.diff(rz[cyl]) > 0).all()
    assert (kinds[dsk] == 1).all() and (np.diff(rz[dsk]) > 0).all()
    # z-extent bounds of "this cylinder and every later one"
    hi = np.array([ls[i]["hi"] for i in cyl], np.float32)
    lo = np.array([ls[i]["lo"] for i in cyl], np.float32)
    assert np.array_equal(outf[1:1 + n_cyl], np.maximum.accumulate(hi[::-1])[::-1])
    assert np.array_equal(outf[65:65 + n_cyl], np.minimum.accumulate(lo[::-1])[::-1])
    assert abs(outf[0] - 0.0029979245800 * 3.8) < 1e-9
    assert out[211] == 1 and out[195] == -1  # one region with every layer (low 32 bits set)


def test_region_masks(lib):
    ls = configs.layer_table("find20")
    plans = [[0, 1, 2, 3], [0, 1, 10, 11], [4, 5]]
    st, out, _ = build(lib, ls, plans, [-1.0, 1.0])
    assert st == MKF_OK and out[211] == 3
    assert out[195] == 0b1111 and out[196] == (1 | 2 | 1 << 10 | 1 << 11) and out[197] == (1 << 4 | 1 << 5)


@pytest.mark.parametrize("bad,code", [
    (dict(kind=2), ERR_GEOMETRY),
    (dict(hi=-130.0), ERR_GEOMETRY),          # hi <= lo
    (dict(sigma_u=0.0), ERR_GEOMETRY),
    (dict(sigma_v=float("nan")), ERR_GEOMETRY),
    (dict(n_phi=0), ERR_GEOMETRY),
    (dict(n_zr=5000), ERR_GEOMETRY),
    (dict(r_or_z=-4.0), ERR_GEOMETRY),        # a cylinder at negative radius
])
def test_invalid_layer_rejected(lib, bad, code):
    ls = [dict(d) for d in configs.layer_table("find20")]
    ls[3].update(bad)
    assert build(lib, ls)[0] == code


def test_invalid_calls_rejected(lib):
    ls = configs.layer_table("find20")
    assert build(lib, ls, bz=float("nan"))[0] == ERR_GEOMETRY
    assert build(lib, ls, [[0, 1], [99]], [0.0])[0] == ERR_GEOMETRY      # plan names a missing layer
    assert build(lib, ls, [[0], [1], [2]], [1.0, 0.5])[0] == ERR_GEOMETRY  # edges not ascending
    assert build(lib, ls * 4)[0] == ERR_CAPACITY                          # more than 64 layers
    huge = [dict(d, n_phi=4096, n_zr=4096) for d in ls[:5]]
    assert build(lib, huge)[0] == ERR_CAPACITY                            # bins per event past 2^26
