"""Runtime helpers around the C ABI: a finding step captured in a CUDA graph,
and autotuners for the finder's launch and the hit-bin grid.

A captured step replays hit binning and finding on fixed device buffers with a
single graph launch; the library performs no allocation or host
synchronisation inside `mkf_hits_bin` / `mkf_find` once a first (warm-up) call
has sized its buffers, which is what makes the capture possible.
"""
from __future__ import annotations

import json
import os

import torch

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")


class CapturedStep:
    """Hit binning + finding on fixed buffers, captured once, replayed many times.

    xyz, layer, event_offsets, seed_hits, seed_event: device tensors whose
    contents may change between replays (sizes may not).  find_kw: mkf_find
    keywords (n_best, chi2_cut, max_out, block_threads, event_times, ...)."""

    def __init__(self, ctx, xyz, layer, event_offsets, seed_hits, seed_event, **find_kw):
        self.ctx = ctx
        self.args = (xyz, layer, event_offsets, seed_hits, seed_event)
        self.kw = find_kw
        self.stream = torch.cuda.Stream(device=xyz.device)
        prev = torch.cuda.current_stream(xyz.device)
        ctx.set_stream(self.stream)
        try:
            with torch.cuda.stream(self.stream):
                self.bins = ctx.hits_bin(xyz, layer, event_offsets)
                self.out = ctx.find(self.bins, seed_hits, seed_event, **find_kw)  # warm-up: sizes all buffers
            self.stream.synchronize()
            ctx.sync()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                ctx.hits_bin(xyz, layer, event_offsets, self.bins)
                ctx.find(self.bins, seed_hits, seed_event, out=self.out, **find_kw)
        finally:
            ctx.set_stream(prev)

    def replay(self):
        self.graph.replay()
        return self.out


def _key(ctx, n_layers, n_best, n_seeds):
    name = torch.cuda.get_device_name(ctx.device)
    bucket = 1 << max(0, int(n_seeds).bit_length() - 1)
    return f"{name}|L{n_layers}|N{n_best}|S{bucket}"


def tune_find_block(ctx, bins, seed_hits, seed_event, n_best=10, candidates=(64, 128, 256), reps=5, cache=True,
                    **find_kw):
    """Time the finder with each block size and return the fastest (cached by
    GPU name, layer count, N and the seed count's power of two)."""
    n_layers = len(ctx.layers) if ctx.layers else 0
    key = _key(ctx, n_layers, n_best, seed_hits.shape[1])
    table = {}
    if cache and os.path.exists(_CACHE):
        try:
            with open(_CACHE) as fh:
                table = json.load(fh)
        except (OSError, ValueError):
            table = {}
    if key in table:
        return int(table[key]["block_threads"]), table[key]
    times = {}
    out = None
    for bt in candidates:
        out = ctx.find(bins, seed_hits, seed_event, n_best=n_best, block_threads=bt, out=out, **find_kw)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            ctx.find(bins, seed_hits, seed_event, n_best=n_best, block_threads=bt, out=out, **find_kw)
        b.record()
        torch.cuda.synchronize()
        times[bt] = a.elapsed_time(b) / reps
    best = min(times, key=times.get)
    rec = {"block_threads": best, "ms": {str(k): v for k, v in times.items()}}
    if cache:
        table[key] = rec
        try:
            with open(_CACHE, "w") as fh:
                json.dump(table, fh, indent=1)
        except OSError:
            pass
    return best, rec


GRIDS = ((128, 16), (256, 16), (256, 32), (512, 32))
BLOCKS = (128, 256)
ORDERS = (0, 1)  # seeds grouped by event and |eta| (the finder's default), input order


def _occupancy_key(ctx, n_layers, n_best, n_seeds, n_hits, n_events):
    name = torch.cuda.get_device_name(ctx.device)
    b = lambda x: 1 << max(0, int(x).bit_length() - 1)
    return (f"{name}|L{n_layers}|N{n_best}|S{b(n_seeds)}|H/ev{b(n_hits // max(1, n_events))}"
            f"|S/ev{b(n_seeds // max(1, n_events))}")


def tune_find_config(ctx, layers, bz, xyz, layer, event_offsets, seed_hits, seed_event, n_best=10, grids=GRIDS,
                     blocks=BLOCKS, orders=ORDERS, reps=3, cache=True, **find_kw):
    """Hit-bin grid (the same n_phi x n_zr on every layer), finder block size
    and seed order of the fastest binning + finding step, timed with CUDA
    events on this workload; cached by GPU, layer count, N, seed count and
    occupancy (hits and seeds per event, powers of two).  Leaves the chosen grid
    loaded in `ctx` (bins made before are then stale) and returns (layers with
    that grid, block size, record with every configuration's time and the
    chosen seed_order)."""
    n_events = event_offsets.shape[0] - 1
    key = "cfg|" + _occupancy_key(ctx, len(layers), n_best, seed_hits.shape[1], xyz.shape[1], n_events)
    table = {}
    if cache and os.path.exists(_CACHE):
        try:
            with open(_CACHE) as fh:
                table = json.load(fh)
        except (OSError, ValueError):
            table = {}
    with_grid = lambda g: [dict(d, n_phi=int(g[0]), n_zr=int(g[1])) for d in layers]
    if key in table:
        rec = table[key]
        ctx.geometry_load(with_grid(rec["grid"]), bz)
        return with_grid(rec["grid"]), int(rec["block_threads"]), rec
    times = {}
    for g in grids:
        ctx.geometry_load(with_grid(g), bz)
        bins = ctx.hits_bin(xyz, layer, event_offsets)
        out = None
        for bt in blocks:
            for so in orders:
                kw = dict(find_kw, block_threads=bt, seed_order=so)
                out = ctx.find(bins, seed_hits, seed_event, n_best=n_best, out=out, **kw)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(reps):
                    ctx.hits_bin(xyz, layer, event_offsets, bins)
                    ctx.find(bins, seed_hits, seed_event, n_best=n_best, out=out, **kw)
                b.record()
                torch.cuda.synchronize()
                times[f"{g[0]}x{g[1]}|{bt}|{so}"] = a.elapsed_time(b) / reps
        del bins, out
    best = min(times, key=times.get)
    gs, bt, so = best.split("|")
    grid = tuple(int(x) for x in gs.split("x"))
    rec = {"grid": list(grid), "block_threads": int(bt), "seed_order": int(so), "ms": times,
           "spread": max(times.values()) / min(times.values()) - 1.0}
    if cache:
        table[key] = rec
        try:
            with open(_CACHE, "w") as fh:
                json.dump(table, fh, indent=1)
        except OSError:
            pass
    ctx.geometry_load(with_grid(grid), bz)
    return with_grid(grid), int(bt), rec
