"""The finder's CUDA source run on the CPU: its device code (seed kernel and
persistent find kernel) compiled for the host with the warp intrinsics emulated
by 32 lane threads that meet at every intrinsic.  It checks the kernel logic --
segmented selection, state hand-off, history walk-back, the first step taken in
the seed kernel -- against the FP64 oracle without a GPU, and that the two
first-step paths give identical results.  (Host arithmetic does not contract
multiply-adds the way the GPU build does: parity holds to the same tolerances,
bit equality is only asserted between two host runs.)"""
import os
import re
import shutil
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import oracle as O
from synth import make_batch
from tests.gpu_helpers import chi2_errors, compare

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1811_04141_gb300", "csrc")


def _device_part(src: str) -> str:
    """The anonymous-namespace part of mkf_find.cu (kernels and helpers) with
    the shared-memory and timer spellings mapped to the host."""
    a = src.index("namespace {")
    b = src.index("}  // namespace") + len("}  // namespace")
    body = src[a:b]
    body = body.replace("extern __shared__ __align__(16) unsigned char smem[];", "unsigned char *smem = g_smem;")
    body = body.replace("__shared__ ", "static ")
    body = re.sub(r'asm volatile\("mov\.u64 %0, %%globaltimer;" : "=l"\(t\)\);', "t = 0;", body)
    return '#include "warp_emu.h"\n#include "mkf_internal.h"\n' + body + "\n"


@pytest.fixture(scope="module")
def emu_so():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    with open(os.path.join(CSRC, "mkf_find.cu")) as f:
        dev = _device_part(f.read())
    with open(os.path.join(d, "find_dev.inc"), "w") as f:
        f.write(dev)
    so = os.path.join(d, "find_emu.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared", "-I" + os.path.join(HERE, "host"),
                    "-I" + d, "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", so,
                    os.path.join(HERE, "host", "find_emu.cpp")], check=True)
    return so


def run_emu(so, cfg, event, n_tracks, n_noise, n_best, step1, mlp_bf16=None, tau=0.0, material=0.0, eloss=0.0,
            alpha=None, gen_field=False, mmap=None):
    d = tempfile.mkdtemp()
    out = os.path.join(d, "out.npz")
    wpath, mpath = "none", "none"
    if mmap is not None:
        mpath = os.path.join(d, "map.npz")
        extra = {} if mmap.get("eloss") is None else {"eloss": mmap["eloss"]}
        np.savez(mpath, r_max=mmap["r_max"], z_min=mmap["z_min"], z_max=mmap["z_max"], x0=mmap["x0"], **extra)
    if mlp_bf16 is not None:
        wpath = os.path.join(d, "w.npy")
        np.save(wpath, mlp_bf16)
    r = subprocess.run([sys.executable, os.path.join(HERE, "host", "run_find_emu.py"), so, cfg, str(event),
                        str(n_tracks), "none" if n_noise is None else str(n_noise), str(n_best), str(step1), out,
                        wpath, str(tau), str(material), str(eloss), "none" if alpha is None else repr(alpha),
                        "1" if gen_field else "0", mpath, ROOT],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    z = np.load(out)
    res = {k: z[k] for k in z.files}
    assert (res["fault"] == 0).all(), res["fault"]
    assert (res["hits"] != -7).all()  # every seed's output row written
    return res


@pytest.mark.parametrize("cfg,event,tracks,noise,n_best", [
    ("find20", 41, 200, None, 1),
    ("find20", 41, 200, None, 10),
    ("dense45", 42, 100, 20000, 16),
])
def test_emulated_finder_matches_oracle(emu_so, cfg, event, tracks, noise, n_best):
    b = make_batch(cfg, [event], n_tracks=tracks, n_noise=noise)
    ref = O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                 n_best=n_best, max_out=len(b.layers) + 3)
    out = run_emu(emu_so, cfg, event, tracks, noise, n_best, 1)
    compare(out, ref)


def test_emulated_seed_phase_precision(emu_so):
    """2000 find20 seeds of an event no other test uses, one of whose chi2
    the seed kernel got 12.5e-3 of max(chi2, ndf) wrong with the seed-hit
    filter's covariance in FP32 entries: with its square root every track
    agrees to half the parity bar."""
    b = make_batch("find20", [30006], n_tracks=2000)
    ref = O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                 n_best=10, max_out=len(b.layers) + 3)
    out = run_emu(emu_so, "find20", 30006, 2000, None, 10, 1)
    compare(out, ref)
    ok = (out["hits"] == ref["hits"]).all(axis=0) & (ref["status"] & O.ST_BADSEED == 0)
    assert ok.sum() > 1950
    assert chi2_errors(out["chi2"][ok], ref["chi2"][ok], 2 * ref["n_hits"][ok] - 5).max() <= 1.0


@pytest.mark.parametrize("n_best,eloss", [(1, 0.0), (10, 0.0), (10, 0.1)])
def test_emulated_finder_with_material_matches_oracle(emu_so, n_best, eloss):
    """The finder variant with material (0.02 X0 in every layer, cylinders and
    disks; scattering, and energy loss when eloss > 0) against the oracle with
    the same material."""
    b = make_batch("find20", [45], n_tracks=150)
    for d in b.layers:
        d["x0"] = 0.02
        d["eloss"] = eloss
    ref = O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                 n_best=n_best, max_out=len(b.layers) + 3)
    out = run_emu(emu_so, "find20", 45, 150, None, n_best, 1, material=0.02, eloss=eloss)
    compare(out, ref)


@pytest.mark.parametrize("cfg,gen_field,n_best", [("fit10", True, 10), ("find20", True, 10), ("find20", False, 1)])
def test_emulated_finder_in_parameterised_field_matches_oracle(emu_so, cfg, gen_field, n_best):
    """The finder variant with Runge-Kutta propagation in the parameterised
    field against the oracle in the same field, on tracks the generator moves
    through that field (fit10; find20, disks too) and, once, on find20 hits
    from the uniform field that only the filter sees in the other one."""
    alpha = 1e-5 if gen_field else 1e-6  # find20's disks reach z = 270 cm
    b = (make_batch(cfg, [46], n_tracks=120, field_alpha=alpha) if gen_field
         else make_batch(cfg, [46], n_tracks=120))
    geo = O.geometry_as_loaded(b, field_alpha=alpha)
    ref = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                 n_best=n_best, max_out=len(b.layers) + 3)
    out = run_emu(emu_so, cfg, 46, 120, None, n_best, 1, alpha=alpha, gen_field=gen_field)
    compare(out, ref)


@pytest.mark.parametrize("n_best", [1, 10])
def test_emulated_finder_with_material_map_matches_oracle(emu_so, n_best):
    """The finder with an r-z material map (each crossing's material from its
    cell) on tracks the generator scatters and slows with the same map."""
    from tests.test_oracle_material_map import _graded_map
    mm = _graded_map()
    b = make_batch("fit10", [47], n_tracks=150, material_map=mm)
    ref = O.find(O.geometry_as_loaded(b), b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                 n_best=n_best, max_out=len(b.layers) + 3)
    out = run_emu(emu_so, "fit10", 47, 150, None, n_best, 1, mmap=mm)
    compare(out, ref)


def test_emulated_first_step_paths_identical(emu_so):
    """First step in the seed kernel vs in the warp: bit-identical on the host."""
    a = run_emu(emu_so, "find20", 43, 50, None, 10, 1)
    w = run_emu(emu_so, "find20", 43, 50, None, 10, 0)
    for k in ("par", "cov", "chi2", "n_hits", "hits", "status", "counters"):
        assert np.array_equal(a[k].view(np.uint32) if a[k].dtype == np.float32 else a[k],
                              w[k].view(np.uint32) if w[k].dtype == np.float32 else w[k]), k


def _bf16_bits(w):
    """float32 -> bfloat16 bit patterns, round to nearest even (the plain definition)."""
    u = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


@pytest.mark.parametrize("tau", [-0.5, 0.5])
def test_emulated_learned_pruning_matches_oracle(emu_so, tau):
    """The finder's learned variant (MLP scores of each candidate's compatible
    hits, pairs below tau dropped before the selection) on the CPU, against the
    oracle with the same bfloat16 weights."""
    from oracle import mlp
    w = mlp.init_weights(21)
    bits = _bf16_bits(w)
    wb = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    b = make_batch("dense45", [44], n_tracks=100, n_noise=200000)
    out = run_emu(emu_so, "dense45", 44, 100, 200000, 10, 1, mlp_bf16=bits, tau=tau)
    geo = O.geometry_as_loaded(b)
    ref = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                 n_best=10, mlp_w=wb, mlp_tau=tau, max_out=len(b.layers) + 3)
    plain = O.find(geo, b.xyz.astype(np.float64), b.layer, b.event_offsets, b.seed_hits, b.seed_event,
                   n_best=10, max_out=len(b.layers) + 3)
    # the network does prune here: fewer updates than the plain finder
    assert ref["counters"][2].sum() < plain["counters"][2].sum()
    same = (out["hits"] == ref["hits"]).all(axis=0)
    m = ref["margins"]
    for k in np.nonzero(~same)[0]:
        assert m[0, k] < 5e-3 or m[1, k] < 2e-3 or m[2, k] < 1e-4 or m[3, k] < 2e-2, (k, m[:, k])
    assert same.mean() >= 0.98
