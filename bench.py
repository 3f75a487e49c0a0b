#!/usr/bin/env python
"""Benchmark of the Kalman-filter finding step on GB300 (one JSON line on stdout).

A step is one pass of the whole finding path over one batch: hit binning
(mkf_hits_bin) and seeded N-best finding (mkf_find: seed state and seed fit,
per-layer propagation, covariance transport, window search, chi2, N-best
selection, Kalman updates, output).  Workload: 20 synthetic events x 2000
tracks, 10 barrel cylinders + 2 x 5 endcap disks in 3.8 T, |eta| < 2.4, 2 %
hit inefficiency, uniform noise at 5x each layer's signal hits, N = 10 best
candidates kept per seed, chi2 cut 30.  Metric: KF candidate-layer updates/s
(one unit = one candidate propagated to one layer and searched).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank processes its own 20 events (weak scaling, no
collective on the data path); rank 0 prints the aggregate.
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
CONFIG = "find20"
EVENTS = 20
N_BEST = 10
CHI2_CUT = 30.0
MAX_CONSEC = 3
WORKLOAD = ("KF track finding, 20 events x 2000 tracks: 10 barrel cylinders r=4..100 cm + 2x5 endcap disks "
            "|z|=120..270 cm, 3.8 T, |eta|<2.4, pT 0.5-10 GeV, 2% hit inefficiency, uniform noise 5x signal "
            "per layer; N=10 best candidates per seed, chi2 cut 30")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle baseline sample")
    ap.add_argument("--events", type=int, default=EVENTS, help="events per GPU (profiling runs only)")
    ap.add_argument("--n-best", type=int, default=N_BEST, help="candidates kept per seed (profiling runs only)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-pruning comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched uneven-events leg")
    ap.add_argument("--batched-events", type=int, default=512)
    ap.add_argument("--no-fit", action="store_true", help="skip the 10^6-track fit leg")
    ap.add_argument("--no-post", action="store_true", help="skip the seed-cleaning / duplicate-removal timing")
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

def oracle_rate(batch, target_s: float):
    """Candidate-layer updates/s of the oracle on a sample of seeds of `batch`,
    sized to take about target_s seconds on one host core."""
    import oracle as O
    geo = O.geometry_as_loaded(batch)
    xyz = batch.xyz.astype(np.float64)
    rng = np.random.default_rng(7)
    order = rng.permutation(batch.n_seeds)
    done, units, t_used = 0, 0, 0.0
    n = 20
    while t_used < target_s and done < batch.n_seeds:
        sel = np.sort(order[done:done + n])
        t0 = time.perf_counter()
        r = O.find(geo, xyz, batch.layer, batch.event_offsets, batch.seed_hits, batch.seed_event, n_best=N_BEST,
                   chi2_cut=CHI2_CUT, max_consec=MAX_CONSEC, seed_list=sel)
        t_used += time.perf_counter() - t0
        units += int(r["counters"][0].sum())
        done += sel.size
        rate = max(t_used, 1e-6) / done
        n = int(min(max(20, (target_s - t_used) / rate), batch.n_seeds - done))
        if n <= 0:
            break
    return units / t_used, done, t_used


# ---------------------------------------------------------------------------
# learned pruning: events/s of the MLP-pruned finder vs the plain finder
# ---------------------------------------------------------------------------

def learned_leg(dev, reps: int = 30):
    """Dense events (17 cylinders + 2 x 14 disks, 6000 tracks + 200k noise hits
    per event): train the MLP on features the plain finder dumps on 10 training
    events (labels from truth), take the largest threshold whose efficiency stays
    within 0.5 points of the plain finder on those events, then time both finders
    (binning + finding) on 10 held-out events."""
    import torch

    from paper_1811_04141_gb300 import Context
    from paper_1811_04141_gb300 import learned as L
    from synth import make_batch
    tr = make_batch("dense45", list(range(1000, 1010)))
    ev = make_batch("dense45", list(range(10)))
    ctx = Context(dev.index, torch.cuda.current_stream(dev))
    ctx.geometry_load(tr.layers, tr.bz)

    def prep(b):
        to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        d = dict(xyz=to(b.xyz, torch.float32), layer=to(b.layer, torch.int32), evo=to(b.event_offsets, torch.int32),
                 sh=to(b.seed_hits, torch.int32), se=to(b.seed_event, torch.int32),
                 hp=to(b.hit_particle, torch.int32), sp=to(b.seed_particle, torch.int32))
        d["bins"] = ctx.hits_bin(d["xyz"], d["layer"], d["evo"])
        return d

    dt, de = prep(tr), prep(ev)
    feat, ref = L.collect_features(ctx, dt["bins"], dt["sh"], dt["se"], 8_000_000, n_best=N_BEST)
    lab = L.label_pairs(ref, dt["hp"], dt["sp"])
    st = L.train(ctx, feat, lab, steps=1500, batch=4096, lr=2e-3)
    max_out = len(tr.layers) + 3

    def run(d, tau=None):
        kw = dict(n_best=N_BEST, max_out=max_out)
        if tau is not None:
            kw.update(mlp_bf16=st["w_bf16"], mlp_tau=tau)
        out = ctx.find(d["bins"], d["sh"], d["se"], **kw)
        ctx.sync()
        e, f = L.efficiency(out["hits"], d["hp"], d["sp"])
        return e, f, out["counters"].sum(dim=1).cpu().numpy()

    e0, f0, _ = run(dt)
    best = L.choose_tau(lambda t: run(dt, t)[:2], e0, [-4.0, -2.0, -1.0, 0.0, 1.0, 2.0, 3.0])
    tau = best[0] if best else None

    def timed(tau_):
        kw = dict(n_best=N_BEST, max_out=max_out)
        if tau_ is not None:
            kw.update(mlp_bf16=st["w_bf16"], mlp_tau=tau_)
        out = ctx.find(de["bins"], de["sh"], de["se"], **kw)
        for _ in range(3):
            ctx.hits_bin(de["xyz"], de["layer"], de["evo"], de["bins"])
            ctx.find(de["bins"], de["sh"], de["se"], out=out, **kw)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            ctx.hits_bin(de["xyz"], de["layer"], de["evo"], de["bins"])
            ctx.find(de["bins"], de["sh"], de["se"], out=out, **kw)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms_plain = timed(None)
    ms_pruned = timed(tau) if tau is not None else None
    ep, fp, cp = run(de)
    # best-hit finding (N = 1) on the same held-out events: what branching buys here
    out1 = ctx.find(de["bins"], de["sh"], de["se"], n_best=1, max_out=max_out)
    for _ in range(3):
        ctx.hits_bin(de["xyz"], de["layer"], de["evo"], de["bins"])
        ctx.find(de["bins"], de["sh"], de["se"], n_best=1, max_out=max_out, out=out1)
    torch.cuda.synchronize()
    a1, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a1.record()
    for _ in range(reps):
        ctx.hits_bin(de["xyz"], de["layer"], de["evo"], de["bins"])
        ctx.find(de["bins"], de["sh"], de["se"], n_best=1, max_out=max_out, out=out1)
    b1.record()
    torch.cuda.synchronize()
    ms_best = a1.elapsed_time(b1) / reps
    e1, f1 = L.efficiency(out1["hits"], de["hp"], de["sp"])
    res = {"workload": "dense45: 17 cylinders + 2x14 disks, 6000 tracks (pT^-3 from 0.5 GeV) + 200k noise hits "
                       "per event; trained on 10 events, evaluated on 10 held-out events; N=10",
           "metric": "events/s (hit binning + finding)", "train_pairs": int(feat.shape[0]),
           "train_loss_first_last": [st["losses"][0], st["losses"][-1]] if st["losses"] else None,
           "plain": {"events_per_s": 10 / (ms_plain * 1e-3), "ms": ms_plain, "efficiency": ep, "fake_rate": fp,
                     "cand_layers": int(cp[0]), "updates": int(cp[2])},
           "best_hit_n1": {"events_per_s": 10 / (ms_best * 1e-3), "ms": ms_best, "efficiency": e1, "fake_rate": f1,
                           "cand_layers": int(out1["counters"][0].sum().item())}}
    if tau is not None:
        el, fl, cl = run(de, tau)
        res["pruned"] = {"tau": tau, "events_per_s": 10 / (ms_pruned * 1e-3), "ms": ms_pruned, "efficiency": el,
                         "fake_rate": fl, "cand_layers": int(cl[0]), "updates": int(cl[2])}
        res["pruned_over_plain_events_per_s"] = ms_plain / ms_pruned
    ctx.close()
    return res


# ---------------------------------------------------------------------------
# batched uneven events in one persistent launch, replayed from a CUDA graph
# ---------------------------------------------------------------------------

def batched_leg(dev, n_events: int = 512, reps: int = 10):
    """Dense geometry, per-event track counts floor(exp(U[ln 100, ln 20000])) and
    noise counts floor(exp(U[ln 1e3, ln 3e5])); the binning + finding step is
    captured in a CUDA graph after choosing the finder's block size; per-event
    latency = time from the finder's first block start until the event's last
    seed is written (GPU global timer)."""
    import torch

    from paper_1811_04141_gb300 import Context
    from paper_1811_04141_gb300.runtime import CapturedStep, tune_find_block
    from synth import make_batch
    rng = np.random.default_rng(4_181_104)
    tracks = np.floor(np.exp(rng.uniform(np.log(100), np.log(20000), n_events))).astype(int)
    noise = np.floor(np.exp(rng.uniform(np.log(1e3), np.log(3e5), n_events))).astype(int)
    t0 = time.perf_counter()
    b = make_batch("dense45", list(range(5000, 5000 + n_events)), n_tracks=list(tracks), n_noise=list(noise))
    gen_s = time.perf_counter() - t0
    ctx = Context(dev.index, torch.cuda.current_stream(dev))
    ctx.geometry_load(b.layers, b.bz)
    to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    xyz, layer, evo = to(b.xyz, torch.float32), to(b.layer, torch.int32), to(b.event_offsets, torch.int32)
    sh, se = to(b.seed_hits, torch.int32), to(b.seed_event, torch.int32)
    max_out = len(b.layers) + 3
    bins = ctx.hits_bin(xyz, layer, evo)
    bt, tune = tune_find_block(ctx, bins, sh, se, n_best=N_BEST, max_out=max_out)
    et = torch.zeros(n_events + 1, dtype=torch.int64, device=dev)
    step = CapturedStep(ctx, xyz, layer, evo, sh, se, n_best=N_BEST, max_out=max_out, block_threads=bt,
                        event_times=et)
    for _ in range(3):
        step.replay()
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        out = step.replay()
    e.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / reps
    t = et.cpu().numpy().astype(np.int64)
    lat_ms = (t[:n_events] - t[n_events]) / 1e6
    cl = int(out["counters"][0].sum().item())
    ctx.close()
    return {"workload": f"{n_events} events, dense geometry (17 cylinders + 2x14 disks), tracks/event "
                        "floor(exp(U[ln 100, ln 20000])), noise/event floor(exp(U[ln 1e3, ln 3e5])), N=10; "
                        "binning + finding replayed from one CUDA graph",
            "events": n_events, "hits": b.n_hits, "seeds": b.n_seeds, "generation_s": round(gen_s, 2),
            "ms_per_replay": ms, "events_per_s": n_events / (ms * 1e-3),
            "cand_layer_updates_per_s": cl / (ms * 1e-3),
            "event_latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                                 "max": float(lat_ms.max())},
            "autotune": {"block_threads": bt, "ms_by_block_threads": tune.get("ms")}}


# ---------------------------------------------------------------------------
# fit: 10^6 tracks along their hit lists
# ---------------------------------------------------------------------------

def fit_leg(dev, n_tracks: int = 1_000_000, reps: int = 20):
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
    peak = flops.fp32_peak_tflops(torch.cuda.get_device_properties(dev).multi_processor_count, 2070.0)
    ctx.close()
    roof = lambda t, k: {"bound": "alu", "achieved": fl / (t * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": fl / (t * 1e-3) / 1e12 / peak, "kernel": k}
    return {"workload": f"{n_ev} events x {n_tracks // n_ev} tracks, 10 barrel cylinders R=4..100 cm, |z|<=125, 3.8 T, |eta|<1, "
                        "pT U[0.5,10] GeV, 20 um / 100 um hits, seeds from the first three hits",
            "track_layer_updates_per_s": layers / (ms * 1e-3), "ms": ms, "roofline": roof(ms, "fit_kernel"),
            "backward": {"workload": "the same tracks fitted in reverse from the forward result at the last hit "
                                     "(covariance x100), state at the first hit",
                         "track_layer_updates_per_s": layers / (ms_b * 1e-3), "ms": ms_b,
                         "roofline": roof(ms_b, "fit_kernel (backward)")}}


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


FIND_DRAM_BYTES = None  # dram__bytes_read.sum + dram__bytes_write.sum of find_kernel on find20; None until re-measured for this kernel version


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


def e2e_pipelined(ctx, batch, bins, NB, max_out, K, W, units_all, pg, dev):
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
                     max_out=max_out, out=d_out[b])
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

def run_ours(args, world, rank, local, pg):
    import torch

    from paper_1811_04141_gb300 import Context, build, flops
    from synth import make_batch

    if local == 0 or world == 1:
        build.build()
    barrier(pg)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1811_04141_gb300.shard import combine, events_for_rank
    E, NB = args.events, args.n_best
    events = events_for_rank(rank, world, E)
    batch = make_batch(CONFIG, events)
    ctx = Context(local, torch.cuda.current_stream(dev))
    ctx.geometry_load(batch.layers, batch.bz)
    to = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    xyz, layer = to(batch.xyz, torch.float32), to(batch.layer, torch.int32)
    evo, sh, se = to(batch.event_offsets, torch.int32), to(batch.seed_hits, torch.int32), to(batch.seed_event,
                                                                                             torch.int32)
    max_out = len(batch.layers) + 3
    bins = ctx.hits_bin(xyz, layer, evo)
    out = ctx.find(bins, sh, se, n_best=NB, chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC, max_out=max_out)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        ctx.hits_bin(xyz, layer, evo, bins)
        ctx.find(bins, sh, se, n_best=NB, chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC, max_out=max_out, out=out)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    ctx.sync()
    cl = int(out["counters"][0].sum().item())
    ht = int(out["counters"][1].sum().item())
    up = int(out["counters"][2].sum().item())

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stream = torch.cuda.current_stream(dev)
    for i in range(K):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        ctx.hits_bin(xyz, layer, evo, bins)
        ev[i][1].record(stream)
        ctx.find(bins, sh, se, n_best=NB, chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC, max_out=max_out,
                 out=out)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ctx.sync()
    step_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in ev]))
    find_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    bin_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    units_all, step_ms_max = combine(pg, cl, step_ms, dev)
    value = units_all / (step_ms_max * 1e-3)

    # roofline of the dominant kernel (find): FP32 ALU bound
    fl = flops.find_flops(cl, ht, up)
    achieved = fl / (find_ms * 1e-3) / 1e12
    peak_mhz = 2070.0
    peak = flops.fp32_peak_tflops(torch.cuda.get_device_properties(dev).multi_processor_count, peak_mhz)
    # DRAM bytes per find_kernel launch on this workload (read + write), from a one-pass ncu
    # capture of the current kernel (profiles/dram.find20_bench.md); only the bench's own
    # workload at the default size has a measured figure
    traffic = FIND_DRAM_BYTES if (E == EVENTS and NB == N_BEST and world >= 1) else None
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": "find_kernel", "kernel_ms": round(find_ms, 4),
                "flops_per_launch": fl, "peak_basis": f"{peak_mhz:.0f} MHz x SMs x 128 FP32 lanes x 2 (derived)"}

    # best-hit finding (N = 1) on the same binned events: a separate object
    best_hit = None
    if rank == 0 and world == 1:
        o1 = ctx.find(bins, sh, se, n_best=1, chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC, max_out=max_out)
        for _ in range(3):
            ctx.find(bins, sh, se, n_best=1, chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC, max_out=max_out, out=o1)
        torch.cuda.synchronize()
        e1 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
        for a, b_ in e1:
            flush.fill_(1.0)
            a.record(stream)
            ctx.find(bins, sh, se, n_best=1, chi2_cut=CHI2_CUT, max_consec_miss=MAX_CONSEC, max_out=max_out, out=o1)
            b_.record(stream)
        torch.cuda.synchronize()
        ms1 = float(np.mean([a.elapsed_time(b_) for a, b_ in e1]))
        cl1 = int(o1["counters"][0].sum().item())
        best_hit = {"workload": "the same 20 events, best-hit finding (N = 1), chi2 cut 30", "find_ms": round(ms1, 4),
                    "step_ms": round(ms1 + bin_ms, 4), "candidate_layers": cl1,
                    "cand_layer_updates_per_s": cl1 / ((ms1 + bin_ms) * 1e-3)}

    # seed cleaning (fit over each seed's three hits + duplicate test) and
    # duplicate-track removal on the step's found tracks: a separate object
    post = None
    if rank == 0 and world == 1 and not args.no_post:
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
        post = {"workload": "the same 20 events: seed cleaning (fit over the 3 seed hits, then the shared-hit and "
                            "(q/pT, eta, phi) duplicate test) and duplicate-track removal on the found tracks "
                            "(shared hits >= half the shorter track)",
                "seed_clean_ms": round(ms_clean, 4), "seeds_per_s": n_seeds / (ms_clean * 1e-3),
                "seeds_removed": int((keep_s == 0).sum().item()),
                "dedup_ms": round(ms_dedup, 4), "tracks_per_s": n_seeds / (ms_dedup * 1e-3),
                "tracks_removed": int((keep_t == 0).sum().item())}

    # end to end through the public API with host buffers: every step copies its
    # inputs from pinned host memory and reads its tracks back; copies run on
    # their own streams, overlapped with the previous / next step's compute
    # (two device buffer sets), as a serving pipeline would run them
    e2e = None
    if not args.no_e2e:
        e2e = e2e_pipelined(ctx, batch, bins, NB, max_out, K, max(3, args.warmup), units_all, pg, dev)
        ctx.set_stream(stream)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, nseeds, secs = oracle_rate(batch, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nseeds} randomly chosen seeds of the {batch.n_seeds} in the workload (all hits of "
                         f"their events), {secs:.1f} s on one host core, FP64"}

    learned = None
    if rank == 0 and world == 1 and not args.no_learned:
        learned = learned_leg(dev)
    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = batched_leg(dev, args.batched_events)
    fit = None
    if rank == 0 and world == 1 and not args.no_fit:
        fit = fit_leg(dev)
    physics = None
    if rank == 0 and world == 1 and args.physics:
        physics = physics_leg(dev)

    launches_per_step = 6  # bin_keys, scan_tiles, scan_write, scatter, seed, find
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(step_ms_max, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if (E, NB) == (EVENTS, N_BEST) else f"{WORKLOAD} [profiling variant: "
                                                                                 f"{E} events, N={NB}]",
                   "events_per_gpu": E, "tracks_per_event": 2000, "n_best": NB,
                   "chi2_cut": CHI2_CUT, "hits_per_gpu": batch.n_hits, "seeds_per_gpu": batch.n_seeds,
                   "cand_layers_per_step_per_gpu": cl, "hits_tested_per_step_per_gpu": ht,
                   "updates_per_step_per_gpu": up, "bin_ms": round(bin_ms, 4), "find_ms": round(find_ms, 4),
                   "l2": "flushed between steps (256 MiB write, outside the per-step CUDA events)",
                   "wall_s_timed_region": round(wall, 3), "parallelism": f"events sharded, {world} GPU(s)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "learned": learned,
        "batched": batched, "fit": fit, "best_hit": best_hit, "post": post, "physics": physics,
        "gpu_launches": launches_per_step * K,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_reference(args, world, rank, local, pg):
    """The FP64 oracle on the host cores, same metric and workload (a bounded
    sample of seeds per step)."""
    if rank != 0:
        return
    from synth import make_batch
    batch = make_batch(CONFIG, list(range(EVENTS)))
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup) * 2)
    for _ in range(args.warmup):
        oracle_rate(batch, per_step / 4)
    rates, seeds, secs = [], 0, 0.0
    for _ in range(args.steps):
        r, n, s = oracle_rate(batch, per_step)
        rates.append(r)
        seeds += n
        secs += s
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events": EVENTS, "tracks_per_event": 2000, "n_best": N_BEST,
                       "chi2_cut": CHI2_CUT},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{seeds} seeds sampled over {args.steps} steps of about {per_step:.1f} s"},
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
