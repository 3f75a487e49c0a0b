#!/usr/bin/env python
"""Benchmark of the Kalman-filter finding step on GB300 (one JSON line on stdout).

A step is one pass of the whole finding path over one batch of events: hit
binning (mkf_hits_bin) and seeded N-best finding (mkf_find: seed state and seed
fit, per-layer propagation, covariance transport, window search, chi2, N-best
selection, Kalman updates, output), replayed from one captured CUDA graph.

Workload (the largest single-GPU configuration): 512 synthetic events of
uneven occupancy on the dense geometry (17 barrel cylinders + 2 x 14 endcap
disks, 3.8 T), per event floor(exp(U[ln 100, ln 20000])) tracks with pT falling
as pT^-3 from 0.5 GeV, |eta| < 2.4, 2 % hit inefficiency, and
floor(exp(U[ln 1e3, ln 3e5])) uniform noise hits; N = 10 best candidates kept per
seed, chi2 cut 30; bin grid, block size and seed order from the autotuner.  Metric: KF
candidate-layer updates/s (one unit = one candidate propagated to one layer and
searched).  Extra objects time the 20-event find20 workload, the fit of 10^6
tracks, learned pruning, seed cleaning and duplicate removal.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank processes its own 512 events (weak scaling,
no collective on the data path); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "KF candidate-layer updates/s"
UNIT = "candidate-layer updates/s"
N_BEST = 10
CHI2_CUT = 30.0
MAX_CONSEC = 3
C4_EVENTS = 512
C4_FIRST_EVENT = 5000
WORKLOAD = ("KF track finding, 512 events of uneven occupancy in one CUDA-graph replay: 17 barrel cylinders + "
            "2x14 endcap disks, 3.8 T, per event floor(exp(U[ln 100, ln 20000])) tracks (pT^-3 from 0.5 GeV, "
            "|eta|<2.4, 2% hit inefficiency) and floor(exp(U[ln 1e3, ln 3e5])) uniform noise hits; N=10 best "
            "candidates per seed, chi2 cut 30, autotuned finder launch")
FIND20 = "find20"
FIND20_EVENTS = 20
FIND20_WORKLOAD = ("KF track finding, 20 events x 2000 tracks: 10 barrel cylinders r=4..100 cm + 2x5 endcap disks "
                   "|z|=120..270 cm, 3.8 T, |eta|<2.4, pT 0.5-10 GeV, 2% hit inefficiency, uniform noise 5x signal "
                   "per layer; N=10 best candidates per seed, chi2 cut 30")


def c4_counts(rank: int):
    """Per-event track and noise counts of the uneven workload's 512 events (rank
    0 draws the same counts as the tests; other ranks their own)."""
    rng = np.random.default_rng(4_181_104 if rank == 0 else [4_181_104, rank])
    tracks = np.floor(np.exp(rng.uniform(np.log(100), np.log(20000), C4_EVENTS))).astype(int)
    noise = np.floor(np.exp(rng.uniform(np.log(1e3), np.log(3e5), C4_EVENTS))).astype(int)
    return tracks, noise


def c4_batch(rank: int, n_events: int = C4_EVENTS, select=None, workers=None):
    """The first n_events of the uneven dense workload of `rank` (event ids
    C4_FIRST_EVENT + rank * 512 onwards), without per-hit truth; `select`: only
    these event positions."""
    from synth import make_batch
    tracks, noise = c4_counts(rank)
    pos = np.arange(min(n_events, C4_EVENTS)) if select is None else np.asarray(select)
    ids = [C4_FIRST_EVENT + rank * C4_EVENTS + int(i) for i in pos]
    return make_batch("dense45", ids, n_tracks=[int(tracks[i]) for i in pos], n_noise=[int(noise[i]) for i in pos],
                      truth=False, workers=workers or os.cpu_count() or 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of each oracle baseline sample (one core, then all cores)")
    ap.add_argument("--events", type=int, default=C4_EVENTS, help="events per GPU (profiling runs only)")
    ap.add_argument("--n-best", type=int, default=N_BEST, help="candidates kept per seed (profiling runs only)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-pruning comparison")
    ap.add_argument("--no-find20", action="store_true", help="skip the 20-event find20 leg")
    ap.add_argument("--no-fit", action="store_true", help="skip the 10^6-track fit leg")
    ap.add_argument("--no-post", action="store_true", help="skip the seed-cleaning / duplicate-removal timing")
    ap.add_argument("--no-peak", action="store_true", help="skip the FP32 peak probe (roofline uses the derived peak)")
    ap.add_argument("--block-threads", type=int, default=0, help="finder block size (0: the autotuner's choice)")
    ap.add_argument("--physics", action="store_true",
                    help="also time the material and parameterised-field fits and the smoother (off by default)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        # each rank on its own GPU before the group exists, so NCCL binds to it
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        import torch
        pg.barrier(device_ids=[torch.cuda.current_device()])


def allreduce_max(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], device="cuda")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], device="cuda")
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------

def _event_slice(batch, e):
    """Hits and seeds of event e as a one-event problem (hit indices made local),
    so that each oracle call scans only that event's hits."""
    lo, hi = int(batch.event_offsets[e]), int(batch.event_offsets[e + 1])
    seeds = np.nonzero(batch.seed_event == e)[0]
    return (np.ascontiguousarray(batch.xyz[:, lo:hi], dtype=np.float64), np.ascontiguousarray(batch.layer[lo:hi]),
            np.array([0, hi - lo], dtype=np.int32), np.ascontiguousarray(batch.seed_hits[:, seeds] - lo),
            np.zeros(seeds.size, dtype=np.int32))


def oracle_rate(batch, target_s: float, threads: int = 1, n_best: int = N_BEST, seed: int = 7):
    """Candidate-layer updates/s of the FP64 oracle on a bounded sample of the
    batch: events in a seeded random order, each event's seeds in chunks of 16,
    the chunks spread over `threads` host threads (the oracle's C code runs
    without the interpreter lock), submitted until about target_s of wall time
    has passed.  Returns (rate, seeds done, events touched, wall seconds)."""
    from concurrent.futures import ThreadPoolExecutor, wait, FIRST_COMPLETED

    import oracle as O
    geo = O.geometry_as_loaded(batch)
    order = np.random.default_rng(seed).permutation(batch.n_events)

    def job(ev, sel):
        x, l, evo, sh, se = ev
        r = O.find(geo, x, l, evo, sh, se, n_best=n_best, chi2_cut=CHI2_CUT, max_consec=MAX_CONSEC, seed_list=sel)
        return int(r["counters"][0].sum()), sel.size

    units = seeds = events = 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        pending = set()
        for e in order:
            ev = _event_slice(batch, int(e))
            n = ev[3].shape[1]
            if n == 0:
                continue
            events += 1
            for c in range(0, n, 16):
                sel = np.arange(c, min(n, c + 16), dtype=np.int64)
                while len(pending) >= 2 * threads:
                    done, pending = wait(pending, return_when=FIRST_COMPLETED)
                    for f in done:
                        u, k = f.result()
                        units, seeds = units + u, seeds + k
                if time.perf_counter() - t0 >= target_s:
                    break
                pending.add(ex.submit(job, ev, sel))
            if time.perf_counter() - t0 >= target_s:
                break
        for f in pending:
            u, k = f.result()
            units, seeds = units + u, seeds + k
    wall = time.perf_counter() - t0
    return units / wall, seeds, events, wall


def cpu_baseline(batch, target_s: float):
    """The oracle on one host core and on all of them (one thread per core)."""
    cores = os.cpu_count() or 1
    r1, s1, e1, w1 = oracle_rate(batch, target_s, 1)
    rn, sn, en, wn = oracle_rate(batch, target_s, cores, seed=8)
    return {"value": rn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sn} seeds of {en} randomly chosen events of the workload (each event's seeds in chunks "
                      f"of 16 over {cores} threads, one per host core), {wn:.1f} s wall, FP64",
            "single_core": {"value": r1, "unit": UNIT, "cores": 1,
                            "sample": f"{s1} seeds of {e1} randomly chosen events, {w1:.1f} s on one host core"}}


def fp32_peak(ctx, dev, iters: int = 50000, reps: int = 5):
    """Measured FP32 rate of the library's FMA-chain probe (TFLOP/s, median of
    `reps` launches timed with CUDA events on the context stream) and the SM
    clock sampled meanwhile."""
    import torch

    from paper_1811_04141_gb300.api import mkf_fp32_probe
    stream = torch.cuda.current_stream(dev)
    out, fl = mkf_fp32_probe(ctx, 100, device=dev)
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, fl = mkf_fp32_probe(ctx, iters, out=out, device=dev)
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    c = clk.stop()
    ms = float(np.median([a.elapsed_time(b) for a, b in ts]))
    return {"tflops": fl / (ms * 1e-3) / 1e12, "ms": round(ms, 3), "flops_per_launch": fl,
            "kernel": "fma_chains_kernel (mkf_fp32_probe: 8 blocks x 256 threads per SM, 8 FMA chains per thread)",
            "clocks": c}


# ---------------------------------------------------------------------------
# learned pruning: events/s of the MLP-pruned finder vs the plain finder
# ---------------------------------------------------------------------------

def learned_leg(dev, n_train: int = 200, n_eval: int = 200, reps: int = 5):
    """Learned branching on dense events (17 cylinders + 2 x 14 disks, 6000 tracks
    + 200k noise hits per event), with material (0.02 X0 and 0.04 GeV per X0 in
    every layer, particles scattered and slowed by the generator) and without.
    The MLP is trained (library kernels) on the pairs the plain N-best finder
    dumps on n_train training events (of the 2000-event training range, events
    0..), labels from truth; the cascade's gate threshold is the smallest that
    keeps efficiency and fake rate within 0.5 points of the plain finder on
    them; timed on n_eval held-out events (10000..): the plain N = 10 finder, the
    learned cascade (best-hit finding with the MLP gate, N-best finding of the
    flagged seeds), the N-best finder with MLP pruning of pairs, and best-hit
    finding; each with hit binning."""
    import torch

    from paper_1811_04141_gb300 import Context
    from paper_1811_04141_gb300 import learned as L
    from synth import make_batch
    res = {"metric": "events/s (hit binning + finding)",
           "training": f"{n_train} of the 2000 training events (0..{n_train - 1}), at most 30M pairs, "
                       "1500 Adam steps of 4096 pairs",
           "evaluation": f"{n_eval} held-out events (10000..{10000 + n_eval - 1})"}
    for kind, mat in (("material", dict(material=0.02, eloss=0.04)), ("clean", {})):
        tr = make_batch("dense45", list(range(n_train)), truth=False, workers=os.cpu_count() or 1, **mat)
        ev = make_batch("dense45", list(range(10000, 10000 + n_eval)), truth=False, workers=os.cpu_count() or 1,
                        **mat)
        ctx = Context(dev.index, torch.cuda.current_stream(dev))
        ctx.geometry_load(tr.layers, tr.bz)
        mo = len(tr.layers) + 3

        def prep(b):
            to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
            d = dict(xyz=to(b.xyz, torch.float32), layer=to(b.layer, torch.int32), evo=to(b.event_offsets, torch.int32),
                     sh=to(b.seed_hits, torch.int32), se=to(b.seed_event, torch.int32),
                     hp=to(b.hit_particle, torch.int32), sp=to(b.seed_particle, torch.int32))
            d["bins"] = ctx.hits_bin(d["xyz"], d["layer"], d["evo"])
            return d

        dt = prep(tr)
        feat, ref = L.collect_features(ctx, dt["bins"], dt["sh"], dt["se"], 30_000_000, n_best=N_BEST, max_out=mo)
        lab = L.label_pairs(ref, dt["hp"], dt["sp"])
        st = L.train(ctx, feat, lab, steps=1500, batch=4096, lr=2e-3)
        del feat, ref, lab

        def eff(d, out):
            return L.efficiency(out["hits"], d["hp"], d["sp"])

        def plain(d, nb=N_BEST, out=None):
            return ctx.find(d["bins"], d["sh"], d["se"], n_best=nb, max_out=mo, out=out)

        def casc(d, tau, out=None, sub=None):
            return L.cascade(ctx, d["bins"], d["sh"], d["se"], st["w_bf16"], tau, n_best=N_BEST, max_out=mo, out=out,
                             subset=sub)

        def pruned(d, tau, out=None):
            return ctx.find(d["bins"], d["sh"], d["se"], n_best=N_BEST, max_out=mo, mlp_bf16=st["w_bf16"],
                            mlp_tau=tau, out=out)

        e0, f0 = eff(dt, plain(dt))
        gate = L.choose_gate_tau(lambda t: eff(dt, casc(dt, t)[0]), e0, f0, [-6.0, -4.0, -2.0, -1.0, 0.0, 1.0, 2.0,
                                                                           3.0, 4.0, 6.0])
        prune = L.choose_tau(lambda t: eff(dt, pruned(dt, t)), e0, [-4.0, -2.0, -1.0, 0.0, 1.0, 2.0, 3.0])
        del dt
        de = prep(ev)

        def timed(fn):
            for _ in range(2):
                ctx.hits_bin(de["xyz"], de["layer"], de["evo"], de["bins"])
                fn()
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                ctx.hits_bin(de["xyz"], de["layer"], de["evo"], de["bins"])
                fn()
            z.record()
            torch.cuda.synchronize()
            return a.elapsed_time(z) / reps

        entry = {}
        o = plain(de)
        ms = timed(lambda: plain(de, out=o))
        e, f = eff(de, o)
        cl = int(o["counters"][0].sum().item())
        entry["plain_n10"] = {"events_per_s": n_eval / (ms * 1e-3), "ms": ms, "efficiency": e, "fake_rate": f,
                              "cand_layers": cl}
        o1 = plain(de, 1)
        ms = timed(lambda: plain(de, 1, out=o1))
        e, f = eff(de, o1)
        entry["best_hit_n1"] = {"events_per_s": n_eval / (ms * 1e-3), "ms": ms, "efficiency": e, "fake_rate": f,
                                "cand_layers": int(o1["counters"][0].sum().item())}
        if gate is not None:
            tau = gate[0]
            oc, sub = casc(de, tau)
            e, f = eff(de, oc)
            flagged = int(sub[1].item())
            ms = timed(lambda: casc(de, tau, out=oc, sub=sub))
            entry["cascade"] = {"tau": tau, "events_per_s": n_eval / (ms * 1e-3), "ms": ms, "efficiency": e,
                                "fake_rate": f, "flagged_seeds": flagged / ev.n_seeds}
            p_ = entry["plain_n10"]
            entry["cascade_over_plain_events_per_s"] = entry["cascade"]["events_per_s"] / p_["events_per_s"]
            entry["cascade_equal_efficiency_and_fake"] = bool(abs(e - p_["efficiency"]) <= 0.005 and
                                                              abs(f - p_["fake_rate"]) <= 0.005)
        if prune is not None:
            tau = prune[0]
            op = pruned(de, tau)
            e, f = eff(de, op)
            ms = timed(lambda: pruned(de, tau, out=op))
            entry["pruned_n10"] = {"tau": tau, "events_per_s": n_eval / (ms * 1e-3), "ms": ms, "efficiency": e,
                                   "fake_rate": f, "cand_layers": int(op["counters"][0].sum().item())}
        entry["train_loss_first_last"] = [st["losses"][0], st["losses"][-1]] if st["losses"] else None
        res[kind] = entry
        ctx.close()
        del de
        torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------------------
# fit: 10^6 tracks along their hit lists
# ---------------------------------------------------------------------------

def fit_leg(dev, peak, n_tracks: int = 1_000_000, reps: int = 20):
    """KF fit of 10^6 tracks (10 barrel cylinders, |eta| < 1, 3.8 T, seeds from the
    first three hits): track-layer updates/s and the fit kernel's FP32 roofline."""
    import torch

    from paper_1811_04141_gb300 import Context, flops
    from synth import make_batch
    n_ev = 5
    b = make_batch("fit10", range(n_ev), n_tracks=n_tracks // n_ev)
    ctx = Context(dev.index, torch.cuda.current_stream(dev))
    ctx.geometry_load(b.layers, b.bz)
    to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    xyz, layer, th = to(b.xyz, torch.float32), to(b.layer, torch.int32), to(b.track_hits, torch.int32)
    out = ctx.fit(xyz, layer, th)
    for _ in range(3):
        ctx.fit(xyz, layer, th, out=out)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    ts = []
    for i in range(reps):
        flush.fill_(float(i))
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.fit(xyz, layer, th, out=out)
        e.record()
        ts.append((a, e))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(e) for a, e in ts]))
    # backward fit of the same tracks from the forward result at the last hit
    outb = ctx.fit_backward(xyz, layer, th, out["par"], out["cov"], 100.0)
    for _ in range(3):
        ctx.fit_backward(xyz, layer, th, out["par"], out["cov"], 100.0, out=outb)
    torch.cuda.synchronize()
    tb = []
    for i in range(reps):
        flush.fill_(float(i))
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.fit_backward(xyz, layer, th, out["par"], out["cov"], 100.0, out=outb)
        e.record()
        tb.append((a, e))
    torch.cuda.synchronize()
    ms_b = float(np.mean([a.elapsed_time(e) for a, e in tb]))
    layers = int((b.track_hits >= 0).sum())
    fl = flops.FLOPS_PER_FIT_LAYER * layers
    # C1 as stated: one event of 1000 tracks, latency of one fit call (launch
    # included), median of 50 back-to-back calls timed one by one
    b1 = make_batch("fit10", [0], n_tracks=1000)
    x1, l1, t1 = to(b1.xyz, torch.float32), to(b1.layer, torch.int32), to(b1.track_hits, torch.int32)
    o1 = ctx.fit(x1, l1, t1)
    for _ in range(5):
        ctx.fit(x1, l1, t1, out=o1)
    torch.cuda.synchronize()
    lat = []
    for _ in range(50):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.fit(x1, l1, t1, out=o1)
        e.record()
        e.synchronize()
        lat.append(a.elapsed_time(e))
    ctx.close()
    roof = lambda t, k: {"bound": "alu", "achieved": fl / (t * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": fl / (t * 1e-3) / 1e12 / peak, "kernel": k}
    return {"workload": f"{n_ev} events x {n_tracks // n_ev} tracks, 10 barrel cylinders R=4..100 cm, |z|<=125, 3.8 T, |eta|<1, "
                        "pT U[0.5,10] GeV, 20 um / 100 um hits, seeds from the first three hits",
            "track_layer_updates_per_s": layers / (ms * 1e-3), "ms": ms, "roofline": roof(ms, "fit_kernel"),
            "backward": {"workload": "the same tracks fitted in reverse from the forward result at the last hit "
                                     "(covariance x100), state at the first hit",
                         "track_layer_updates_per_s": layers / (ms_b * 1e-3), "ms": ms_b,
                         "roofline": roof(ms_b, "fit_kernel (backward)")},
            "c1_latency": {"workload": "1 event x 1000 tracks (fit10), one mkf_fit call",
                           "ms_median": float(np.median(lat)), "ms_p90": float(np.percentile(lat, 90))}}


def physics_leg(dev, n_events: int = 5, per_event: int = 10000, reps: int = 10):
    """Timing of the fit's physics variants on fit10 tracks (off by default,
    --physics): the material variant (0.03 X0 and 0.04 GeV/X0 per layer, tracks
    scattered and slowed by the generator), the parameterised-field variant
    (alpha = 1e-5 /cm^2, tracks moved through that field by the generator) and
    the smoother (state at every hit, inflate 100) on uniform-field tracks."""
    import torch

    from paper_1811_04141_gb300 import Context
    from synth import make_batch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for i in range(reps):
            flush.fill_(float(i))
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            e.record()
            ts.append((a, e))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(e) for a, e in ts]))

    res = {}
    cases = (("material", dict(material=0.03, eloss=0.04), "fit"),
             ("field", dict(field_alpha=1e-5), "fit"),
             ("smoother", {}, "smooth"))
    for name, kw, kind in cases:
        b = make_batch("fit10", range(n_events), n_tracks=per_event, **kw)
        ctx = Context(dev.index, torch.cuda.current_stream(dev))
        ctx.geometry_load(b.layers, b.bz, field_alpha=b.meta.get("field_alpha"))
        xyz, layer, th = to(b.xyz, torch.float32), to(b.layer, torch.int32), to(b.track_hits, torch.int32)
        if kind == "fit":
            out = ctx.fit(xyz, layer, th)
            ms = timed(lambda: ctx.fit(xyz, layer, th, out=out))
        else:
            out = ctx.fit_smooth(xyz, layer, th)
            ms = timed(lambda: ctx.fit_smooth(xyz, layer, th, out=out))
        ctx.close()
        layers = int((b.track_hits >= 0).sum())
        res[name] = {"tracks": int(b.n_seeds), "ms": ms, "track_layer_updates_per_s": layers / (ms * 1e-3)}
    return res


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one mkf_find call
# (seed_kernel, the order's scan and scatter, find_kernel) per candidate-layer it
# processes, from a one-pass ncu capture of the current kernels on 96 of the 512
# uneven dense events (the whole workload exceeds the capture size rule): 618.4 MB
# for 46.5 M candidate-layers (the finder's ncu summary under profiles/); the traffic
# (hit records, seed records, outputs) grows with the candidate-layers processed.
FIND_DRAM_BYTES_PER_CAND_LAYER = 13.30


def _carve(arena, specs):
    """Typed views into one byte arena: specs = [(name, dtype, shape)], each view
    256-byte aligned.  Returns (views, bytes used)."""
    import torch
    views, off = {}, 0
    for name, dt, shape in specs:
        n = int(np.prod(shape)) * torch.empty(0, dtype=dt).element_size()
        views[name] = arena[off:off + n].view(dt).view(*shape)
        off += (n + 255) // 256 * 256
    return views, off


def e2e_pipelined(ctx, batch, bins, NB, max_out, K, W, units_all, pg, dev, find_kw=None):
    """Host -> device copy of the step's inputs (one pinned arena, one copy),
    binning + finding, device -> host copy of all its outputs (one arena, one
    copy); three streams, two device buffer sets, events between the stages.
    Timed from the first timed step's input copy to its last read-back, on the
    device; the working set of two steps in flight (~190 MB) exceeds the L2, and
    every step's inputs arrive fresh from the host."""
    import torch
    n, S, E = batch.n_hits, batch.n_seeds, len(batch.event_offsets) - 1
    in_specs = [("xyz", torch.float32, (3, n)), ("layer", torch.int32, (n,)), ("evo", torch.int32, (E + 1,)),
                ("sh", torch.int32, (3, S)), ("se", torch.int32, (S,))]
    out_specs = [("par", torch.float32, (6, S)), ("cov", torch.float32, (21, S)), ("chi2", torch.float32, (S,)),
                 ("n_hits", torch.int32, (S,)), ("hits", torch.int32, (max_out, S)), ("status", torch.int32, (S,)),
                 ("counters", torch.int32, (3, S))]
    size = lambda specs: sum((int(np.prod(sh)) * torch.empty(0, dtype=dt).element_size() + 255) // 256 * 256
                             for _, dt, sh in specs)
    in_bytes, out_bytes = size(in_specs), size(out_specs)
    h_in_arena = torch.empty(in_bytes, dtype=torch.uint8).pin_memory()
    h_in, _ = _carve(h_in_arena, in_specs)
    for k, arr in (("xyz", batch.xyz), ("layer", batch.layer), ("evo", batch.event_offsets), ("sh", batch.seed_hits),
                   ("se", batch.seed_event)):
        h_in[k].copy_(torch.as_tensor(np.ascontiguousarray(arr)))
    h_out_arena = torch.empty(out_bytes, dtype=torch.uint8).pin_memory()
    d_in_arena = [torch.empty(in_bytes, dtype=torch.uint8, device=dev) for _ in range(2)]
    d_out_arena = [torch.empty(out_bytes, dtype=torch.uint8, device=dev) for _ in range(2)]
    d_in = [_carve(a, in_specs)[0] for a in d_in_arena]
    d_out = [_carve(a, out_specs)[0] for a in d_out_arena]
    s_in, s_comp, s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in", "comp", "out")}
    ctx.set_stream(s_comp)

    def step(i):
        b = i % 2
        if i >= 2:
            s_in.wait_event(ev["comp"][b])
        with torch.cuda.stream(s_in):
            d_in_arena[b].copy_(h_in_arena, non_blocking=True)
            ev["in"][b].record(s_in)
        s_comp.wait_event(ev["in"][b])
        if i >= 2:
            s_comp.wait_event(ev["out"][b])
        with torch.cuda.stream(s_comp):
            x = d_in[b]
            ctx.hits_bin(x["xyz"], x["layer"], x["evo"], bins)
            ctx.find(bins, x["sh"], x["se"], n_best=NB, chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC,
                     max_out=max_out, out=d_out[b], **(find_kw or {}))
            ev["comp"][b].record(s_comp)
        s_out.wait_event(ev["comp"][b])
        with torch.cuda.stream(s_out):
            h_out_arena.copy_(d_out_arena[b], non_blocking=True)
            ev["out"][b].record(s_out)

    for i in range(W):
        step(i)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(s_in)
    for i in range(W, W + K):
        step(i)
    t1.record(s_out)
    torch.cuda.synchronize()
    # the copied-back tracks are the device's
    assert torch.equal(h_out_arena, d_out_arena[(W + K - 1) % 2].cpu())
    ms = allreduce_max(pg, t0.elapsed_time(t1) / K)
    return {"value": units_all / (ms * 1e-3), "unit": UNIT, "ms_per_step": round(ms, 4),
            "h2d_bytes_per_step": int(sum(v.numel() * v.element_size() for v in h_in.values())),
            "d2h_bytes_per_step": int(sum(v.numel() * v.element_size() for v in d_out[0].values())), "copies": "1 H2D + 1 D2H per step on their own streams, "
            "overlapped with the neighbouring steps' compute (2 device buffer sets)"}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------

def find20_leg(dev, peak_tflops, steps: int = 50, config: str = FIND20, events=None, workload=FIND20_WORKLOAD):
    """A fixed-size finding workload (binning + N = 10 finding, eager launches,
    L2 flushed between steps) and best-hit finding (N = 1) on the same events:
    by default find20 (20 events x 2000 tracks); bin grid, block size and seed
    order from the autotuner for each."""
    import torch

    from paper_1811_04141_gb300 import Context, flops
    from paper_1811_04141_gb300.runtime import tune_find_config
    from synth import make_batch
    batch = make_batch(config, list(range(FIND20_EVENTS)) if events is None else list(events), truth=False,
                       workers=os.cpu_count() or 1)
    ctx = Context(dev.index, torch.cuda.current_stream(dev))
    ctx.geometry_load(batch.layers, batch.bz)
    to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    xyz, layer = to(batch.xyz, torch.float32), to(batch.layer, torch.int32)
    evo, sh, se = to(batch.event_offsets, torch.int32), to(batch.seed_hits, torch.int32), to(batch.seed_event,
                                                                                             torch.int32)
    max_out = len(batch.layers) + 3
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {"workload": workload, "events": batch.n_events, "hits": batch.n_hits, "seeds": batch.n_seeds}
    for nb in (N_BEST, 1):
        # bin grid, block size and seed order from the autotuner for this
        # workload and N (it leaves the chosen grid loaded)
        fkw = dict(chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC, max_out=max_out)
        _, bt, tune = tune_find_config(ctx, batch.layers, batch.bz, xyz, layer, evo, sh, se, n_best=nb, **fkw)
        fkw.update(block_threads=bt, seed_order=tune.get("seed_order", 0))
        bins = ctx.hits_bin(xyz, layer, evo)
        out = ctx.find(bins, sh, se, n_best=nb, **fkw)
        for _ in range(3):
            ctx.hits_bin(xyz, layer, evo, bins)
            ctx.find(bins, sh, se, n_best=nb, out=out, **fkw)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            ctx.hits_bin(xyz, layer, evo, bins)
            ev[i][1].record(stream)
            ctx.find(bins, sh, se, n_best=nb, out=out, **fkw)
            ev[i][2].record(stream)
        torch.cuda.synchronize()
        ctx.sync()
        step_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in ev]))
        find_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
        cl, ht, up = (int(out["counters"][i].sum().item()) for i in range(3))
        fl = flops.find_flops(cl, ht, up)
        res["n_best_%d" % nb] = {
            "cand_layer_updates_per_s": cl / (step_ms * 1e-3), "step_ms": round(step_ms, 4),
            "bin_ms": round(step_ms - find_ms, 4), "find_ms": round(find_ms, 4), "candidate_layers": cl,
            "hits_tested": ht, "updates": up,
            "roofline": {"bound": "alu", "achieved": fl / (find_ms * 1e-3) / 1e12, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": fl / (find_ms * 1e-3) / 1e12 / peak_tflops,
                         "kernel": "mkf_find (seed_kernel + find_kernel)"},
            "autotune": {"grid": tune.get("grid"), "block_threads": bt, "seed_order": tune.get("seed_order", 0),
                         "spread": tune.get("spread")}}
    ctx.close()
    return res


def run_ours(args, world, rank, local, pg):
    import torch

    from paper_1811_04141_gb300 import Context, build, flops
    from paper_1811_04141_gb300.runtime import CapturedStep, tune_find_config

    if local == 0 or world == 1:
        build.build()
    # the workload is generated (in spawned processes) before any GPU work
    t0 = time.perf_counter()
    batch = c4_batch(rank, args.events)
    gen_s = time.perf_counter() - t0
    barrier(pg)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1811_04141_gb300.shard import combine
    NB = args.n_best
    E = batch.n_events
    ctx = Context(local, torch.cuda.current_stream(dev))
    ctx.geometry_load(batch.layers, batch.bz)
    to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    xyz, layer = to(batch.xyz, torch.float32), to(batch.layer, torch.int32)
    evo, sh, se = to(batch.event_offsets, torch.int32), to(batch.seed_hits, torch.int32), to(batch.seed_event,
                                                                                             torch.int32)
    max_out = len(batch.layers) + 3
    fkw = dict(chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC, max_out=max_out)

    # measured FP32 peak (the roofline's denominator)
    peak = None
    if not args.no_peak:
        peak = fp32_peak(ctx, dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    derived = flops.fp32_peak_tflops(sm_count, 2070.0)
    peak_tflops = peak["tflops"] if peak else derived

    # hit-bin grid and finder launch from the autotuner (cached per GPU,
    # geometry, size and occupancy)
    if args.block_threads:
        bt, tune = args.block_threads, {"ms": None, "fixed": True, "grid": None, "seed_order": 0}
    else:
        _, bt, tune = tune_find_config(ctx, batch.layers, batch.bz, xyz, layer, evo, sh, se, n_best=NB, **fkw)
    bins = ctx.hits_bin(xyz, layer, evo)
    fkw["block_threads"] = bt
    fkw["seed_order"] = tune.get("seed_order", 0)

    # eager launches with events between the stages: binning and mkf_find times
    out = ctx.find(bins, sh, se, n_best=NB, **fkw)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(2):
        ctx.hits_bin(xyz, layer, evo, bins)
        ctx.find(bins, sh, se, n_best=NB, out=out, **fkw)
    torch.cuda.synchronize()
    n_eager = 5
    eg = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_eager)]
    for i in range(n_eager):
        flush.fill_(float(i))
        eg[i][0].record(stream)
        ctx.hits_bin(xyz, layer, evo, bins)
        eg[i][1].record(stream)
        ctx.find(bins, sh, se, n_best=NB, out=out, **fkw)
        eg[i][2].record(stream)
    torch.cuda.synchronize()
    ctx.sync()
    bin_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in eg]))
    find_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in eg]))
    cl = int(out["counters"][0].sum().item())
    ht = int(out["counters"][1].sum().item())
    up = int(out["counters"][2].sum().item())

    # the timed step: binning + finding of all events, one CUDA-graph replay
    et = torch.zeros(E + 1, dtype=torch.int64, device=dev)
    step = CapturedStep(ctx, xyz, layer, evo, sh, se, n_best=NB, event_times=et, **fkw)
    gs = step.stream
    with torch.cuda.stream(gs):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step.replay()
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    lat = []
    clocks = ClockSampler(local)
    clocks.start()
    barrier(pg)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    with torch.cuda.stream(gs):
        for i in range(K):
            flush.fill_(float(i))  # inputs (~0.9 GB) exceed the L2 anyway; the flush keeps outputs out too
            ev[i][0].record(gs)
            o = step.replay()
            ev[i][1].record(gs)
    torch.cuda.synchronize()
    barrier(pg)
    wall = time.perf_counter() - w0
    clk = clocks.stop()
    ctx.sync()
    t = et.cpu().numpy().astype(np.int64)
    lat_ms = (t[:E] - t[E]) / 1e6
    step_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    cl_g = int(o["counters"][0].sum().item())
    assert cl_g == cl, (cl_g, cl)  # the replay does the same work as the eager launches
    units_all, step_ms_max = combine(pg, cl, step_ms, dev)
    value = units_all / (step_ms_max * 1e-3)

    # roofline of the dominant launch (mkf_find: seed_kernel + find_kernel), FP32 ALU bound
    fl = flops.find_flops(cl, ht, up)
    achieved = fl / (find_ms * 1e-3) / 1e12
    traffic = (None if FIND_DRAM_BYTES_PER_CAND_LAYER is None or NB != N_BEST
               else int(FIND_DRAM_BYTES_PER_CAND_LAYER * cl))
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak_tflops, 4), "traffic": traffic,
                "kernel": "mkf_find (seed_kernel + find_kernel)", "kernel_ms": round(find_ms, 4),
                "flops_per_launch": fl,
                "peak_basis": ("measured: mkf_fp32_probe (FMA chains) on this GPU, median of 5 launches"
                               if peak else f"derived: {sm_count} SMs x 128 FP32 lanes x 2 x 2070 MHz"),
                "derived_peak": round(derived, 2), "fp32_probe": peak}

    e2e = None
    if not args.no_e2e:
        e2e = e2e_pipelined(ctx, batch, bins, NB, max_out, K, max(3, args.warmup), units_all, pg, dev,
                            find_kw={"block_threads": bt, "seed_order": fkw["seed_order"]})
        ctx.set_stream(stream)
    ctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(batch, args.cpu_seconds)
    extras = {}
    if rank == 0 and world == 1:
        if not args.no_find20:
            extras["find20"] = find20_leg(dev, peak_tflops)
            extras["dense50"] = find20_leg(
                dev, peak_tflops, steps=10, config="dense45", events=range(50),
                workload="KF track finding, 50 dense events x 6000 tracks (pT^-3 from 0.5 GeV) + 200k uniform noise "
                         "hits: 17 barrel cylinders + 2x14 endcap disks, |eta|<2.4, 2% hit inefficiency; N=10, chi2 "
                         "cut 30")
        if not args.no_fit:
            extras["fit"] = fit_leg(dev, peak_tflops)
        if not args.no_post:
            extras["post"] = post_leg(dev)
        if not args.no_learned:
            extras["learned"] = learned_leg(dev)
        if args.physics:
            extras["physics"] = physics_leg(dev)

    launches_per_step = 8  # bin_keys, scan_tiles, scan_write, scatter, seed, where_scan, order_scatter, find
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(step_ms_max, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if (E, NB) == (C4_EVENTS, N_BEST) else f"{WORKLOAD} [profiling variant: "
                                                                                  f"{E} events, N={NB}]",
                   "events_per_gpu": E, "n_best": NB, "chi2_cut": CHI2_CUT, "hits_per_gpu": batch.n_hits,
                   "seeds_per_gpu": batch.n_seeds, "cand_layers_per_step_per_gpu": cl,
                   "hits_tested_per_step_per_gpu": ht, "updates_per_step_per_gpu": up,
                   "bin_ms_eager": round(bin_ms, 4), "find_ms_eager": round(find_ms, 4),
                   "events_per_s": units_all / cl * E / (step_ms_max * 1e-3),
                   "event_latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                                        "p99": float(np.percentile(lat_ms, 99)), "max": float(lat_ms.max()),
                                        "basis": "GPU global timer at each event's last seed output, from the "
                                                 "finder's first block"},
                   "launch": "binning + finding captured in one CUDA graph, replayed per step",
                   "autotune": {"grid": tune.get("grid"), "block_threads": bt, "seed_order": fkw["seed_order"],
                                "ms_by_grid_and_block": tune.get("ms"), "spread": tune.get("spread")},
                   "l2": "inputs (~0.9 GB) larger than L2, and a 256 MiB write between steps outside the events",
                   "generation_s": round(gen_s, 1), "wall_s_timed_region": round(wall, 3),
                   "parallelism": f"events sharded, {world} GPU(s)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "gpu_launches": launches_per_step * K,
    }
    line.update(extras)
    if rank == 0:
        print(json.dumps(line), flush=True)


def post_leg(dev):
    """Seed cleaning (fit over each seed's three hits + duplicate test) and
    duplicate-track removal on the find20 step's 40 k seeds and found tracks."""
    import torch

    from paper_1811_04141_gb300 import Context
    from synth import make_batch
    batch = make_batch(FIND20, list(range(FIND20_EVENTS)))
    ctx = Context(dev.index, torch.cuda.current_stream(dev))
    ctx.geometry_load(batch.layers, batch.bz)
    to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    xyz, layer = to(batch.xyz, torch.float32), to(batch.layer, torch.int32)
    evo, sh, se = to(batch.event_offsets, torch.int32), to(batch.seed_hits, torch.int32), to(batch.seed_event,
                                                                                             torch.int32)
    bins = ctx.hits_bin(xyz, layer, evo)
    out = ctx.find(bins, sh, se, n_best=N_BEST, max_out=len(batch.layers) + 3)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b_ in e2:
            flush.fill_(1.0)
            a.record(stream)
            fn()
            b_.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b_) for a, b_ in e2]))

    sfit = ctx.fit(xyz, layer, sh)
    keep_s = ctx.seeds_clean(sh, batch.n_hits, sfit["par"])
    keep_t = ctx.tracks_dedup(out["hits"], batch.n_hits, out["n_hits"], out["chi2"])
    ms_clean = timed(lambda: (ctx.fit(xyz, layer, sh, out=sfit),
                              ctx.seeds_clean(sh, batch.n_hits, sfit["par"], keep=keep_s)))
    ms_dedup = timed(lambda: ctx.tracks_dedup(out["hits"], batch.n_hits, out["n_hits"], out["chi2"], keep=keep_t))
    n_seeds = int(sh.shape[1])
    res = {"workload": "find20 (20 events x 2000 tracks): seed cleaning (fit over the 3 seed hits, then the "
                       "shared-hit and (q/pT, eta, phi) duplicate test) and duplicate-track removal on the found "
                       "tracks (shared hits >= half the shorter track)",
           "seed_clean_ms": round(ms_clean, 4), "seeds_per_s": n_seeds / (ms_clean * 1e-3),
           "seeds_removed": int((keep_s == 0).sum().item()),
           "dedup_ms": round(ms_dedup, 4), "tracks_per_s": n_seeds / (ms_dedup * 1e-3),
           "tracks_removed": int((keep_t == 0).sum().item())}
    ctx.close()
    return res


def run_reference(args, world, rank, local, pg):
    """The FP64 oracle on the host cores (one thread per core), same metric and
    workload: each step a bounded sample of the uneven dense events.  Under
    torchrun only rank 0 runs it."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    # the sampled events only (events are independent and seeded by their id)
    sel = np.random.default_rng(11).choice(C4_EVENTS, 24, replace=False)
    batch = c4_batch(0, select=np.sort(sel))
    per_step = max(0.5, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup):
        oracle_rate(batch, per_step / 4, cores, seed=100 + i)
    rates, seeds, secs = [], 0, 0.0
    for i in range(args.steps):
        r, n, _, w = oracle_rate(batch, per_step, cores, seed=200 + i)
        rates.append(r)
        seeds += n
        secs += w
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_gpu": C4_EVENTS, "n_best": N_BEST, "chi2_cut": CHI2_CUT},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{seeds} seeds of 24 of the workload's events sampled over {args.steps} "
                                       f"steps of about {per_step:.1f} s, {cores} threads (one per host core)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local, pg = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank, local, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
