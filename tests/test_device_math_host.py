"""CPU checks of self-contained helpers of the device math header, compiled for
the host with the same FP32 expressions: the bounded-range sin/cos against
float64 sin/cos, and the sinc series against its closed form."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1811_04141_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "devmath.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + CSRC, "-o", so,
                    os.path.join(HERE, "host", "device_math_host.cpp")], check=True)
    return C.CDLL(so)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def test_sincos_small_accuracy(lib):
    rng = np.random.default_rng(0)
    x = _f32(np.concatenate([np.linspace(-8, 8, 400001), rng.uniform(-1e-3, 1e-3, 20000),
                             np.array([0.0, np.pi / 2, np.pi, -np.pi, 3 * np.pi / 2, 2 * np.pi, 1e-30, -1e-30])]))
    s = np.empty_like(x)
    c = np.empty_like(x)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    lib.host_sincos_small(p(x), p(s), p(c), x.size)
    xs = x.astype(np.float64)
    es, ec = np.abs(s - np.sin(xs)), np.abs(c - np.cos(xs))
    ulp1 = np.spacing(np.float32(1.0))
    # absolute error within two float ulps of 1, relative within three ulps
    assert es.max() <= 2 * ulp1 and ec.max() <= 2 * ulp1, (es.max(), ec.max())
    big_s, big_c = np.abs(np.sin(xs)) > 1e-3, np.abs(np.cos(xs)) > 1e-3
    assert (es[big_s] / np.abs(np.sin(xs))[big_s]).max() <= 3 * ulp1
    assert (ec[big_c] / np.abs(np.cos(xs))[big_c]).max() <= 3 * ulp1
    # odd / even symmetry and sin^2 + cos^2
    sm, cm = np.empty_like(x), np.empty_like(x)
    xm = _f32(-x)
    lib.host_sincos_small(p(xm), p(sm), p(cm), x.size)
    assert np.array_equal(sm, -s) and np.array_equal(cm, c)
    assert np.abs(s.astype(np.float64) ** 2 + c.astype(np.float64) ** 2 - 1).max() <= 4 * ulp1


def test_sinc_series_matches_closed_form(lib):
    a = _f32(np.concatenate([np.linspace(-1.5, 1.5, 30001), np.array([0.0, 0.2499, 0.25, -0.25])]))
    sn, dsn = np.empty_like(a), np.empty_like(a)
    p = lambda v: v.ctypes.data_as(C.c_void_p)
    lib.host_sinc_and_deriv(p(a), p(sn), p(dsn), a.size)
    ad = a.astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = np.where(ad == 0, 1.0, np.sin(ad) / ad)
        dref = np.where(ad == 0, 0.0, (ad * np.cos(ad) - np.sin(ad)) / ad ** 2)
    assert np.abs(sn - ref).max() <= 3e-7
    assert np.abs(dsn - dref).max() <= 3e-6
