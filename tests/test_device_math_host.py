"""CPU checks of self-contained helpers of the device math header, compiled for
the host with the same FP32 expressions: the bounded-range sin/cos against
float64 sin/cos, the sinc series against its closed form, and the square-root
form of the seed-hit filter (prior, transport, material, Potter update) against
the closed-form prior and the covariance form of the Kalman filter."""
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


# ---- the square-root form of the seed-hit filter

KB = 3.8 * 0.0029979245800
NSQ = 9  # square-root columns of the host build


def _sym(c21):
    m = np.zeros((6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            m[i, j] = m[j, i] = c21[k]
            k += 1
    return m


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def test_square_root_seed_prior(lib):
    """S S^T of the seed prior's square root equals the prior's closed form:
    variance sigma^2 along the first layer's surface and none along its normal,
    (0.1 q/pT)^2 + 1e-4 on q/pT, 1e-4 on phi and on theta, nothing else."""
    s2 = np.float32(0.02 ** 2)
    cases = [(0, [4.0 * np.cos(0.7), 4.0 * np.sin(0.7), 3.1], [14.5 * np.cos(0.76), 14.5 * np.sin(0.76), 11.0],
              [25.1 * np.cos(0.85), 25.1 * np.sin(0.85), 19.4]),
             (1, [30.0, -12.0, 120.0], [37.0, -16.5, 157.5], [44.5, -21.5, 195.0])]
    for kind, h1, h2, h3 in cases:
        h1, h2, h3 = _f32(h1), _f32(h2), _f32(h3)
        par, cov = np.zeros(6, np.float32), np.zeros(21, np.float32)
        k = lib.host_seed_prior(kind, C.c_float(s2), C.c_float(KB), _p(h1), _p(h2), _p(h3), _p(par), _p(cov))
        assert k == 5
        ref = np.zeros((6, 6))
        if kind == 0:
            a = np.arctan2(float(h1[1]), float(h1[0]))
            t = np.array([-np.sin(a), np.cos(a), 0.0])
            ref[:3, :3] = float(s2) * (np.outer(t, t) + np.diag([0.0, 0.0, 1.0]))
        else:
            ref[0, 0] = ref[1, 1] = float(s2)
        ref[3, 3] = (0.1 * float(par[3])) ** 2 + 1e-4
        ref[4, 4] = ref[5, 5] = 1e-4
        assert np.allclose(_sym(cov), ref, rtol=1e-6, atol=1e-12), (kind, _sym(cov) - ref)


def _kalman64(S, par, kind, su2, sv2, u, v):
    """The textbook update in float64 on C = S S^T: K = C H^T (H C H^T + V)^-1."""
    Cm = S.astype(np.float64) @ S.astype(np.float64).T
    x, y = float(par[0]), float(par[1])
    r = np.hypot(x, y)
    cp, sp = x / r, y / r
    H = np.zeros((2, 6))
    H[0, 0], H[0, 1] = -sp, cp
    if kind == 0:
        H[1, 2] = 1.0
    else:
        H[1, 0], H[1, 1] = cp, sp
    Sm = H @ Cm @ H.T + np.diag([su2, sv2])
    Si = np.linalg.inv(Sm)
    K = Cm @ H.T @ Si
    res = np.array([u, v])
    return Cm - K @ H @ Cm, K @ res, float(res @ Si @ res), H, Cm


def test_potter_update_matches_kalman_update(lib):
    """One hit through the square root (two scalar Potter steps) equals the
    2-D Kalman update in float64 on C = S S^T: covariance, state change and
    chi2, on cylinders and disks."""
    lib.host_sqrt_update.restype = C.c_float
    rng = np.random.default_rng(11)
    scale = np.array([3e-3, 3e-3, 5e-3, 2e-2, 1e-3, 1e-3])
    for trial in range(200):
        kind = trial % 2
        S = _f32(rng.normal(size=(6, NSQ)) * scale[:, None])
        a = rng.uniform(-np.pi, np.pi)
        par = _f32([4.0 * np.cos(a), 4.0 * np.sin(a), rng.uniform(-10, 10), rng.uniform(-2, 2),
                    rng.uniform(-np.pi, np.pi), rng.uniform(0.5, 2.6)])
        su2, sv2 = (2e-3) ** 2, (1e-2) ** 2 if kind == 0 else (2e-3) ** 2
        u, v = rng.normal(scale=3e-3), rng.normal(scale=1e-2)
        Cn, dp, chi2, _, Cm = _kalman64(S, par, kind, su2, sv2, u, v)
        S2, p2 = S.copy().ravel(), par.copy()
        c = lib.host_sqrt_update(kind, C.c_float(su2), C.c_float(sv2), _p(S2), _p(p2), C.c_float(u), C.c_float(v))
        S2 = S2.reshape(6, NSQ).astype(np.float64)
        assert np.abs(S2 @ S2.T - Cn).max() <= 2e-5 * np.abs(Cm).max()
        assert np.abs((p2.astype(np.float64) - par.astype(np.float64)) - dp).max() <= 1e-4 * np.abs(dp).max() + 2e-6
        assert abs(c - chi2) <= 2e-5 * max(chi2, 1.0)


def test_potter_update_keeps_what_fp32_entries_lose(lib):
    """A prior ~1e7 times wider than the hit variance: the square root keeps the
    measured directions' posterior, H C' H^T = V - V S^-1 V, to 3e-3; the same
    update in FP32 covariance entries (C - K H C) misses it by orders more."""
    rng = np.random.default_rng(5)
    worst_sqrt, worst_plain = 0.0, 0.0
    for trial in range(50):
        S = _f32(rng.normal(size=(6, NSQ)) * np.array([2.0, 2.0, 2.0, 0.1, 0.5, 0.5])[:, None])
        a = rng.uniform(-np.pi, np.pi)
        par = _f32([4.0 * np.cos(a), 4.0 * np.sin(a), 1.0, 0.5, a, 1.2])
        su2 = sv2 = (2e-3) ** 2
        Cn, dp, chi2, H, Cm = _kalman64(S, par, 0, su2, sv2, 0.0, 0.0)
        exact = H @ Cn @ H.T
        S2, p2 = S.copy().ravel(), par.copy()
        lib.host_sqrt_update(0, C.c_float(su2), C.c_float(sv2), _p(S2), _p(p2), C.c_float(0.0), C.c_float(0.0))
        S2 = S2.reshape(6, NSQ).astype(np.float64)
        got = H @ (S2 @ S2.T) @ H.T
        worst_sqrt = max(worst_sqrt, np.abs(got - exact).max() / np.abs(exact).max())
        # the short form in FP32 entries
        C32, H32 = Cm.astype(np.float32), H.astype(np.float32)
        Sm32 = H32 @ C32 @ H32.T + np.diag(np.float32([su2, sv2]))
        K32 = C32 @ H32.T @ np.linalg.inv(Sm32).astype(np.float32)
        Cn32 = (C32 - K32 @ (H32 @ C32)).astype(np.float64)
        worst_plain = max(worst_plain, np.abs(H @ Cn32 @ H.T - exact).max() / np.abs(exact).max())
    assert worst_sqrt <= 3e-3, worst_sqrt
    assert worst_plain >= 30 * worst_sqrt, (worst_plain, worst_sqrt)


def test_square_root_transport_matches_covariance(lib):
    """The move onto a cylinder and onto a disk: S' S'^T with S' = J S equals
    J C J^T of the covariance path."""
    rng = np.random.default_rng(2)
    n = 0
    for trial in range(100):
        kind = trial % 2
        S = _f32(rng.normal(size=(6, NSQ)) * np.array([3e-3, 3e-3, 5e-3, 2e-2, 1e-3, 1e-3])[:, None])
        a = rng.uniform(-np.pi, np.pi)
        th = rng.uniform(0.3, 1.2) if kind == 1 else rng.uniform(0.6, 2.5)
        par = _f32([4.0 * np.cos(a), 4.0 * np.sin(a), 2.0, rng.choice([-1, 1]) * rng.uniform(0.1, 1.5),
                    a + rng.uniform(-0.3, 0.3), th])
        cc, cs = np.zeros(21, np.float32), np.zeros(21, np.float32)
        ok = lib.host_transport_both(kind, C.c_float(25.0 if kind == 0 else 120.0), C.c_float(KB), _p(par), _p(S.ravel().copy()),
                                     _p(cc), _p(cs))
        if not ok:
            continue
        n += 1
        assert np.abs(cs.astype(np.float64) - cc).max() <= 1e-5 * np.abs(cc).max(), (kind, trial)
    assert n >= 60


def test_square_root_material_matches_noise(lib):
    """Scattering noise appended as two columns and the energy loss applied to
    the q/pT row give the covariance path's C + Q and F C F^T."""
    rng = np.random.default_rng(4)
    for trial in range(100):
        kind = trial % 2
        used = 5 if trial % 4 < 2 else 7
        S = rng.normal(size=(6, NSQ)) * np.array([3e-3, 3e-3, 5e-3, 2e-2, 1e-3, 1e-3])[:, None]
        S[:, used:] = 0.0
        S = _f32(S)
        a = rng.uniform(-np.pi, np.pi)
        par = _f32([25.0 * np.cos(a), 25.0 * np.sin(a), 10.0, rng.choice([-1, 1]) * rng.uniform(0.1, 2.0),
                    a + rng.uniform(-0.3, 0.3), rng.uniform(0.4, 2.7)])
        cc, cs = np.zeros(21, np.float32), np.zeros(21, np.float32)
        lib.host_material_both(kind, C.c_float(0.02), C.c_float(0.04), _p(par), _p(S.ravel().copy()), used, _p(cc), _p(cs))
        base = _sym(_sym_pack(S))
        assert np.abs(_sym(cc) - base).max() > 0.0  # the material changed C
        assert np.abs(cs.astype(np.float64) - cc).max() <= 1e-6 * np.abs(cc).max(), (kind, used, trial)


def _sym_pack(S):
    m = S.astype(np.float64) @ S.astype(np.float64).T
    return np.array([m[i, j] for i in range(6) for j in range(i + 1)])
