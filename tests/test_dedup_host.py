"""CPU check of the seed-cleaning and duplicate-removal kernels of mkf_dedup.cu,
compiled for the host and run thread by thread, against the oracle
(oracle/dedup.py): keep flags identical on random lists and on overlap events."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
import oracle.dedup as D
from synth import make_batch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1811_04141_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "mkf_dedup.cu")).read()
    a = src.index("namespace {")
    b = src.index("// Inverse index hit -> items of `lists`")
    body = src[a:b] + "\n}  // namespace\n"
    d = tempfile.mkdtemp()
    with open(os.path.join(d, "dedup_dev.inc"), "w") as f:
        f.write('#include "mkf_internal.h"\n' + body)
    so = os.path.join(d, "dedup_emu.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(HERE, "host"), "-I" + d,
                    "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", so,
                    os.path.join(HERE, "host", "dedup_emu.cpp")], check=True)
    return C.CDLL(so)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _seeds(lib, sh, n_hits, par, tol):
    sh = np.ascontiguousarray(sh, dtype=np.int32)
    par = np.ascontiguousarray(par, dtype=np.float32)
    keep = np.full(sh.shape[1], -1, dtype=np.int32)
    lib.emu_seeds_clean(_p(sh), sh.shape[1], int(n_hits), _p(par), *(C.c_float(x) for x in tol), _p(keep))
    return keep


def _tracks(lib, hidx, n_hits, nh, c2, f):
    hidx = np.ascontiguousarray(hidx, dtype=np.int32)
    nh = np.ascontiguousarray(nh, dtype=np.int32)
    c2 = np.ascontiguousarray(c2, dtype=np.float32)
    keep = np.full(hidx.shape[1], -1, dtype=np.int32)
    lib.emu_tracks_dedup(_p(hidx), hidx.shape[0], hidx.shape[1], int(n_hits), _p(nh), _p(c2), C.c_float(f), _p(keep))
    return keep


@pytest.mark.parametrize("seed", range(3))
def test_kernels_match_oracle_random(lib, seed):
    rng = np.random.default_rng(100 + seed)
    n, n_hits = 777, 300
    sh = rng.integers(-3, n_hits + 5, size=(3, n))
    par = np.zeros((6, n), np.float32)
    par[3] = rng.choice([-1.0, 1.0], n) * rng.uniform(0.1, 0.3, n)
    par[4] = rng.uniform(-np.pi, np.pi, n)
    par[5] = rng.uniform(0.2, 2.9, n)
    for tol in ((0.5, 0.02, 0.02), (0.1, 1.0, 1.5), (0.0, 0.0, 0.0)):
        assert (_seeds(lib, sh, n_hits, par, tol).astype(bool) == D.clean_seeds(sh, n_hits, par, *tol)).all(), tol
    hidx = rng.integers(-2, n_hits + 2, size=(9, n))
    hidx[4] = hidx[2]
    nh = rng.integers(3, 10, n)
    c2 = rng.integers(0, 3, n).astype(np.float32)
    for f in (0.0, 0.25, 0.5, 1.0):
        assert (_tracks(lib, hidx, n_hits, nh, c2, f).astype(bool) == D.dedup_tracks(hidx, n_hits, nh, c2, f)).all(), f


def test_kernels_match_oracle_overlap_events(lib):
    b = make_batch("find20", [5], n_tracks=250, overlap=0.15)
    geo = O.geometry_as_loaded(b)
    par = O.fit(geo, b.xyz.astype(np.float64), b.layer, b.seed_hits)["par"].astype(np.float32)
    keep = _seeds(lib, b.seed_hits, b.n_hits, par, (0.5, 0.02, 0.02))
    assert (keep.astype(bool) == D.clean_seeds(b.seed_hits, b.n_hits, par)).all()
    assert (keep.astype(bool) == (b.seed_dup_of < 0)).all()
    r = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event, n_best=10,
               max_out=len(b.layers) + 3)
    c2 = r["chi2"].astype(np.float32)
    keep = _tracks(lib, r["hits"], b.n_hits, r["n_hits"], c2, 0.5)
    assert (keep.astype(bool) == D.dedup_tracks(r["hits"], b.n_hits, r["n_hits"], c2, 0.5)).all()
