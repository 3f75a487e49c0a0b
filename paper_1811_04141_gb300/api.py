"""Python binding of the C ABI with the same names (mkf_create, mkf_geometry_load,
mkf_hits_bin, mkf_fit, mkf_fit_backward, mkf_fit_smooth, mkf_seeds_clean, mkf_tracks_dedup, mkf_find, mkf_sync,
mkf_destroy), plus a small Context
class.  PyTorch supplies device memory and streams; this module only checks
tensor shapes, dtypes and devices and passes raw pointers to libmkf.so.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need(t, name, dtype, shape=None, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def mkf_create(device: int = 0, stream=None):
    """Create a library context on `device` enqueueing on `stream` (a
    torch.cuda.Stream, a raw cudaStream_t int, or None = torch's current stream)."""
    if stream is None:
        stream = torch.cuda.current_stream(device)
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    h = C.c_void_p()
    N.check("mkf_create", N.lib().mkf_create(C.byref(h), int(device), C.c_void_p(raw)))
    return h


def mkf_destroy(ctx) -> None:
    N.lib().mkf_destroy(ctx)


def mkf_set_stream(ctx, stream) -> None:
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    N.check("mkf_set_stream", N.lib().mkf_set_stream(ctx, C.c_void_p(raw)))


def mkf_sync(ctx) -> None:
    N.check("mkf_sync", N.lib().mkf_sync(ctx))


def mkf_geometry_load(ctx, layers, bz: float, plans=None, region_eta_edges=None, field_alpha=None,
                      material_map=None) -> None:
    """layers: list of dicts (kind, r_or_z, lo, hi, sigma_u, sigma_v, n_phi, n_zr,
    optional x0 = material in radiation lengths); plans: list of layer-id lists,
    one per region (None = one region, all layers); field_alpha: None for the
    uniform field, else the parameterised field's fall-off (1/cm^2);
    material_map: None, or an r-z map dict (r_max, z_min, z_max, x0 [nr, nz],
    eloss [nr, nz] or None)."""
    arr = (N.MkfLayer * len(layers))()
    for i, d in enumerate(layers):
        arr[i] = N.MkfLayer(int(d["kind"]), float(d["r_or_z"]), float(d["lo"]), float(d["hi"]),
                            float(d["sigma_u"]), float(d["sigma_v"]), int(d.get("n_phi", 64)), int(d.get("n_zr", 8)))
    n_plans = 0 if plans is None else len(plans)
    parr, keep, edges = None, [], None
    if n_plans:
        parr = (N.MkfPlan * n_plans)()
        for r, ids in enumerate(plans):
            a = (C.c_int32 * max(1, len(ids)))(*[int(x) for x in ids])
            keep.append(a)
            parr[r] = N.MkfPlan(len(ids), C.cast(a, C.POINTER(C.c_int32)))
        e = list(region_eta_edges or [])
        if len(e) != n_plans - 1:
            raise ValueError("need n_plans - 1 region edges")
        edges = (C.c_float * max(1, len(e)))(*[float(x) for x in e])
    N.check("mkf_geometry_load", N.lib().mkf_geometry_load(
        ctx, arr, len(layers), parr, n_plans, edges, float(bz)))
    if any(float(d.get("x0", 0.0)) > 0.0 for d in layers):
        mkf_geometry_material(ctx, [float(d.get("x0", 0.0)) for d in layers],
                              [float(d.get("eloss", 0.0)) for d in layers])
    if field_alpha is not None:
        mkf_geometry_field(ctx, 1, field_alpha)
    if material_map is not None:
        mkf_geometry_material_map(ctx, material_map["x0"], material_map["r_max"], material_map["z_min"],
                                  material_map["z_max"], material_map.get("eloss"))


def mkf_geometry_material(ctx, x0, eloss=None) -> None:
    """Per-layer material of the loaded geometry: x0 in radiation lengths at
    normal incidence, eloss the mean energy loss per radiation length (GeV) or
    None (layer dicts passed to mkf_geometry_load may carry them as "x0" and
    "eloss")."""
    arr = (C.c_float * max(1, len(x0)))(*[float(v) for v in x0])
    earr = None if eloss is None else (C.c_float * max(1, len(eloss)))(*[float(v) for v in eloss])
    N.check("mkf_geometry_material", N.lib().mkf_geometry_material(ctx, arr, earr, len(x0)))


def mkf_geometry_field(ctx, kind: int, alpha: float = 0.0) -> None:
    """Field type of the loaded geometry: 0 uniform, 1 parameterised
    (Bz = bz (1 - alpha (z^2 - r^2 / 2)), Br = bz alpha r z; alpha in 1/cm^2)."""
    N.check("mkf_geometry_field", N.lib().mkf_geometry_field(ctx, int(kind), float(alpha)))


def mkf_geometry_material_map(ctx, x0, r_max: float, z_min: float, z_max: float, eloss=None) -> None:
    """r-z material map of the loaded geometry: x0 and eloss arrays [nr, nz]
    over [0, r_max) x [z_min, z_max); x0 = None removes the map."""
    if x0 is None:
        N.check("mkf_geometry_material_map", N.lib().mkf_geometry_material_map(ctx, 0, 0, 1.0, 0.0, 1.0, None, None))
        return
    import numpy as np
    a = np.ascontiguousarray(x0, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("x0 must be [nr, nz]")
    e = None if eloss is None else np.ascontiguousarray(eloss, dtype=np.float32)
    if e is not None and e.shape != a.shape:
        raise ValueError("eloss must have the shape of x0")
    N.check("mkf_geometry_material_map", N.lib().mkf_geometry_material_map(
        ctx, a.shape[0], a.shape[1], float(r_max), float(z_min), float(z_max), a.ctypes.data,
        None if e is None else e.ctypes.data))


class HitBins:
    """Library-owned bin store; freed with the object (or explicitly)."""

    def __init__(self):
        self.handle = C.c_void_p()

    def info(self) -> dict:
        nh, ne, nb = C.c_int32(), C.c_int32(), C.c_int64()
        N.check("mkf_hitbins_info", N.lib().mkf_hitbins_info(self.handle, C.byref(nh), C.byref(ne), C.byref(nb)))
        return dict(n_hits=nh.value, n_events=ne.value, n_bins=nb.value)

    def export(self, ctx, device="cuda") -> dict:
        """Copies of the store's arrays: rec [n_hits, 4] float32, inv [n_hits] int32,
        offsets [n_bins + 1] int32 (on the context's stream)."""
        i = self.info()
        rec = torch.empty(i["n_hits"], 4, dtype=torch.float32, device=device)
        inv = torch.empty(i["n_hits"], dtype=torch.int32, device=device)
        off = torch.empty(i["n_bins"] + 1, dtype=torch.int32, device=device)
        h = ctx.handle if hasattr(ctx, "handle") else ctx
        N.check("mkf_hitbins_export", N.lib().mkf_hitbins_export(h, self.handle, _ptr(rec), _ptr(inv), _ptr(off)))
        return dict(rec=rec, inv=inv, offsets=off, **i)

    def free(self):
        if self.handle:
            N.lib().mkf_hitbins_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mkf_hits_bin(ctx, xyz, layer, event_offsets, bins: HitBins | None = None, device: int | None = None) -> HitBins:
    n = xyz.shape[1]
    _need(xyz, "xyz", torch.float32, (3, n), device)
    _need(layer, "layer", torch.int32, (n,), device)
    _need(event_offsets, "event_offsets", torch.int32, None, device)
    n_events = event_offsets.shape[0] - 1
    bins = bins or HitBins()
    N.check("mkf_hits_bin", N.lib().mkf_hits_bin(ctx, _ptr(xyz), _ptr(layer), _ptr(event_offsets), n_events, n,
                                                 C.byref(bins.handle)))
    return bins


def mkf_hits_bin_static(ctx, xyz, layer, event_offsets, rec, inv, offsets, device: int | None = None) -> None:
    """Binning into caller-owned buffers with no GPU allocation (for callers that
    cannot allocate device memory); rec [n_hits, 4] float32, inv [n_hits] int32,
    offsets [n_bins + 1] int32, filled like HitBins.export()."""
    n = xyz.shape[1]
    _need(xyz, "xyz", torch.float32, (3, n), device)
    _need(layer, "layer", torch.int32, (n,), device)
    _need(event_offsets, "event_offsets", torch.int32, None, device)
    _need(rec, "rec", torch.float32, (n, 4), device)
    _need(inv, "inv", torch.int32, (n,), device)
    _need(offsets, "offsets", torch.int32, None, device)
    layers = getattr(ctx, "layers", None)
    if layers:
        # every one of the n_bins + 1 entries is written on the device
        n_bins = (event_offsets.shape[0] - 1) * sum(int(d.get("n_phi", 64)) * int(d.get("n_zr", 8)) for d in layers)
        if offsets.numel() != n_bins + 1:
            raise ValueError(f"offsets must have n_bins + 1 = {n_bins + 1} entries, got {offsets.numel()}")
    h = ctx.handle if hasattr(ctx, "handle") else ctx
    N.check("mkf_hits_bin_static", N.lib().mkf_hits_bin_static(
        h, _ptr(xyz), _ptr(layer), _ptr(event_offsets), event_offsets.shape[0] - 1, n, _ptr(rec), _ptr(inv),
        _ptr(offsets)))


def mkf_fit(ctx, xyz, hit_layer, hit_idx, seed_par=None, seed_cov=None, out=None, device: int | None = None):
    """Fit along fixed hit lists; returns dict(par [6,n], cov [21,n], chi2, ndf, status)."""
    n_hits = xyz.shape[1]
    _need(xyz, "xyz", torch.float32, (3, n_hits), device)
    _need(hit_layer, "hit_layer", torch.int32, (n_hits,), device)
    max_hits, n = hit_idx.shape
    _need(hit_idx, "hit_idx", torch.int32, (max_hits, n), device)
    if (seed_par is None) != (seed_cov is None):
        raise ValueError("give both seed_par and seed_cov or neither")
    if seed_par is not None:
        _need(seed_par, "seed_par", torch.float32, (6, n), device)
        _need(seed_cov, "seed_cov", torch.float32, (21, n), device)
    dev = xyz.device
    if out is None:
        out = dict(par=torch.empty(6, n, device=dev), cov=torch.empty(21, n, device=dev),
                   chi2=torch.empty(n, device=dev), ndf=torch.empty(n, dtype=torch.int32, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev))
    N.check("mkf_fit", N.lib().mkf_fit(ctx, _ptr(xyz), _ptr(hit_layer), n_hits, _ptr(hit_idx), max_hits, n,
                                       _ptr(seed_par), _ptr(seed_cov), _ptr(out["par"]), _ptr(out["cov"]),
                                       _ptr(out["chi2"]), _ptr(out["ndf"]), _ptr(out["status"])))
    return out


def mkf_fit_backward(ctx, xyz, hit_layer, hit_idx, last_par, last_cov, inflate=100.0, out=None,
                     device: int | None = None):
    """Backward fit along fixed hit lists (path order) from the state at each
    track's last hit; returns dict(par [6,n], cov [21,n], chi2, ndf, status) at
    the first hit."""
    n_hits = xyz.shape[1]
    _need(xyz, "xyz", torch.float32, (3, n_hits), device)
    _need(hit_layer, "hit_layer", torch.int32, (n_hits,), device)
    max_hits, n = hit_idx.shape
    _need(hit_idx, "hit_idx", torch.int32, (max_hits, n), device)
    _need(last_par, "last_par", torch.float32, (6, n), device)
    _need(last_cov, "last_cov", torch.float32, (21, n), device)
    dev = xyz.device
    if out is None:
        out = dict(par=torch.empty(6, n, device=dev), cov=torch.empty(21, n, device=dev),
                   chi2=torch.empty(n, device=dev), ndf=torch.empty(n, dtype=torch.int32, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev))
    N.check("mkf_fit_backward", N.lib().mkf_fit_backward(
        ctx, _ptr(xyz), _ptr(hit_layer), n_hits, _ptr(hit_idx), max_hits, n, _ptr(last_par), _ptr(last_cov),
        C.c_float(inflate), _ptr(out["par"]), _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out["ndf"]),
        _ptr(out["status"])))
    return out


def mkf_fit_smooth(ctx, xyz, hit_layer, hit_idx, seed_par=None, seed_cov=None, inflate=100.0, out=None,
                   device: int | None = None):
    """Smoothed state at every hit of fixed hit lists (path order): dict(par
    [max_hits, 6, n], cov [max_hits, 21, n] per row of hit_idx, NaN where none;
    chi2, ndf, status of the forward fit)."""
    n_hits = xyz.shape[1]
    _need(xyz, "xyz", torch.float32, (3, n_hits), device)
    _need(hit_layer, "hit_layer", torch.int32, (n_hits,), device)
    max_hits, n = hit_idx.shape
    _need(hit_idx, "hit_idx", torch.int32, (max_hits, n), device)
    if (seed_par is None) != (seed_cov is None):
        raise ValueError("give both seed_par and seed_cov or neither")
    if seed_par is not None:
        _need(seed_par, "seed_par", torch.float32, (6, n), device)
        _need(seed_cov, "seed_cov", torch.float32, (21, n), device)
    dev = xyz.device
    if out is None:
        out = dict(par=torch.empty(max_hits, 6, n, device=dev), cov=torch.empty(max_hits, 21, n, device=dev),
                   chi2=torch.empty(n, device=dev), ndf=torch.empty(n, dtype=torch.int32, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev))
    N.check("mkf_fit_smooth", N.lib().mkf_fit_smooth(
        ctx, _ptr(xyz), _ptr(hit_layer), n_hits, _ptr(hit_idx), max_hits, n,
        None if seed_par is None else _ptr(seed_par), None if seed_cov is None else _ptr(seed_cov),
        C.c_float(inflate), _ptr(out["par"]), _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out["ndf"]),
        _ptr(out["status"])))
    return out


def mkf_seeds_clean(ctx, seed_hits, n_hits, seed_par, max_dqpt=0.5, max_deta=0.02, max_dphi=0.02, keep=None,
                    device: int | None = None):
    """keep [n_seeds] int32 (1 = keep, 0 = duplicate of a lower-index seed)."""
    n = seed_hits.shape[1]
    _need(seed_hits, "seed_hits", torch.int32, (3, n), device)
    _need(seed_par, "seed_par", torch.float32, (6, n), device)
    if keep is None:
        keep = torch.empty(n, dtype=torch.int32, device=seed_hits.device)
    N.check("mkf_seeds_clean", N.lib().mkf_seeds_clean(ctx, _ptr(seed_hits), n, int(n_hits), _ptr(seed_par),
                                                       C.c_float(max_dqpt), C.c_float(max_deta), C.c_float(max_dphi),
                                                       _ptr(keep)))
    return keep


def mkf_tracks_dedup(ctx, hit_idx, n_hits, track_nhits, chi2, min_frac=0.5, keep=None, device: int | None = None):
    """keep [n] int32 (1 = keep, 0 = a better duplicate exists)."""
    max_hits, n = hit_idx.shape
    _need(hit_idx, "hit_idx", torch.int32, (max_hits, n), device)
    _need(track_nhits, "track_nhits", torch.int32, (n,), device)
    _need(chi2, "chi2", torch.float32, (n,), device)
    if keep is None:
        keep = torch.empty(n, dtype=torch.int32, device=hit_idx.device)
    N.check("mkf_tracks_dedup", N.lib().mkf_tracks_dedup(ctx, _ptr(hit_idx), max_hits, n, int(n_hits),
                                                         _ptr(track_nhits), _ptr(chi2), C.c_float(min_frac),
                                                         _ptr(keep)))
    return keep


def find_params(n_best=10, chi2_cut=30.0, max_consec_miss=3, block_threads=0, mlp_bf16=None, mlp_tau=0.0,
                feat=None, event_times=None, seed_list=None, seed_count=None, mlp_mode=0,
                seed_order=0) -> N.MkfFindParams:
    prm = N.MkfFindParams(int(n_best), float(chi2_cut), int(max_consec_miss), int(block_threads))
    if seed_list is not None:
        prm.seed_list = seed_list.data_ptr()
        prm.seed_count = seed_count.data_ptr()
    prm.mlp_mode = int(mlp_mode)
    prm.seed_order = int(seed_order)
    if event_times is not None:
        prm.event_times = event_times.data_ptr()
    if mlp_bf16 is not None:
        prm.mlp_bf16 = mlp_bf16.data_ptr()
        prm.mlp_tau = float(mlp_tau)
    if feat is not None:
        prm.feat_out = feat["feat"].data_ptr()
        prm.feat_ref = feat["ref"].data_ptr()
        prm.feat_count = feat["count"].data_ptr()
        prm.feat_cap = int(feat["feat"].shape[0])
    return prm


def feature_buffer(cap: int, device="cuda") -> dict:
    """Device buffers for the finder's feature dump (counter zeroed)."""
    return dict(feat=torch.empty(cap, N.MLP_IN, device=device), ref=torch.empty(cap, 3, dtype=torch.int32, device=device),
                count=torch.zeros(1, dtype=torch.int32, device=device))


def mkf_find(ctx, bins: HitBins, seed_hits, seed_event, n_best=10, chi2_cut=30.0, max_consec_miss=3, max_out=None,
             n_layers=None, out=None, counters=True, block_threads=0, device: int | None = None, mlp_bf16=None,
             mlp_tau=0.0, feat=None, event_times=None, seed_list=None, seed_count=None, mlp_mode=0, seed_order=0):
    """Find tracks; returns dict(par, cov, chi2, n_hits, hits [max_out, n], status, counters [3, n]).
    mlp_bf16 (int16 tensor of MLP_PARAMS bfloat16 patterns) turns on learned pruning at mlp_tau
    (mlp_mode 1: the gate, flagging seeds instead of dropping hits); feat (from feature_buffer)
    receives the features of every compatible hit; seed_list / seed_count (int32 device
    tensors, the count of one element) restrict the call to those seeds (outputs in `out`
    at their indices)."""
    if (seed_list is None) != (seed_count is None):
        raise ValueError("give both seed_list and seed_count or neither")
    if seed_list is not None:
        _need(seed_list, "seed_list", torch.int32, None, device)
        _need(seed_count, "seed_count", torch.int32, (1,), device)
    n = seed_hits.shape[1]
    _need(seed_hits, "seed_hits", torch.int32, (3, n), device)
    _need(seed_event, "seed_event", torch.int32, (n,), device)
    if mlp_bf16 is not None:
        _need(mlp_bf16, "mlp_bf16", torch.int16, (N.MLP_PARAMS,), device)
    if feat is not None:
        _need(feat["feat"], "feat", torch.float32, None, device)
        _need(feat["ref"], "feat ref", torch.int32, None, device)
        _need(feat["count"], "feat count", torch.int32, (1,), device)
    if max_out is None:
        max_out = (n_layers or N.MAX_LAYERS) + 3
    dev = seed_hits.device
    if out is None:
        out = dict(par=torch.empty(6, n, device=dev), cov=torch.empty(21, n, device=dev),
                   chi2=torch.empty(n, device=dev), n_hits=torch.empty(n, dtype=torch.int32, device=dev),
                   hits=torch.empty(max_out, n, dtype=torch.int32, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev),
                   counters=torch.empty(3, n, dtype=torch.int32, device=dev) if counters else None)
    if event_times is not None:
        _need(event_times, "event_times", torch.int64, None, device)
    prm = find_params(n_best, chi2_cut, max_consec_miss, block_threads, mlp_bf16, mlp_tau, feat, event_times,
                      seed_list, seed_count, mlp_mode, seed_order)
    N.check("mkf_find", N.lib().mkf_find(_h(ctx), bins.handle, _ptr(seed_hits), _ptr(seed_event), n, C.byref(prm),
                                         _ptr(out["par"]), _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out["n_hits"]),
                                         _ptr(out["hits"]), int(out["hits"].shape[0]), _ptr(out["status"]),
                                         _ptr(out.get("counters"))))
    return out


def mkf_seeds_where(ctx, status, bits, seed_list=None, seed_count=None):
    """Indices of the seeds whose status has any of `bits` (device list and a
    one-element device count, both written on the device)."""
    n = status.shape[0]
    _need(status, "status", torch.int32, (n,), None)
    if seed_list is None:
        seed_list = torch.empty(max(1, n), dtype=torch.int32, device=status.device)
    if seed_count is None:
        seed_count = torch.empty(1, dtype=torch.int32, device=status.device)
    N.check("mkf_seeds_where", N.lib().mkf_seeds_where(_h(ctx), _ptr(status), n, int(bits), _ptr(seed_list),
                                                         _ptr(seed_count)))
    return seed_list, seed_count


def _h(ctx):
    return ctx.handle if hasattr(ctx, "handle") else ctx


def mkf_mlp_to_bf16(ctx, w, out=None):
    """FP32 weights -> bfloat16 bit patterns (int16 tensor)."""
    _need(w, "w", torch.float32)
    out = torch.empty(w.shape, dtype=torch.int16, device=w.device) if out is None else out
    N.check("mkf_mlp_to_bf16", N.lib().mkf_mlp_to_bf16(_h(ctx), _ptr(w), _ptr(out), w.numel()))
    return out


def mkf_mlp_forward(ctx, w_bf16, feat, out=None):
    n = feat.shape[0]
    _need(w_bf16, "w_bf16", torch.int16, (N.MLP_PARAMS,))
    _need(feat, "feat", torch.float32, (n, N.MLP_IN))
    out = torch.empty(n, device=feat.device) if out is None else out
    N.check("mkf_mlp_forward", N.lib().mkf_mlp_forward(_h(ctx), _ptr(w_bf16), _ptr(feat), n, _ptr(out)))
    return out


def mkf_mlp_grad(ctx, w_bf16, feat, label):
    n = feat.shape[0]
    _need(w_bf16, "w_bf16", torch.int16, (N.MLP_PARAMS,))
    _need(feat, "feat", torch.float32, (n, N.MLP_IN))
    _need(label, "label", torch.float32, (n,))
    grad = torch.empty(N.MLP_PARAMS, device=feat.device)
    loss = torch.empty(1, device=feat.device)
    N.check("mkf_mlp_grad", N.lib().mkf_mlp_grad(_h(ctx), _ptr(w_bf16), _ptr(feat), _ptr(label), n, _ptr(grad),
                                                 _ptr(loss)))
    return grad, loss


def mkf_fp32_probe(ctx, iters: int, out=None, device=None):
    """Enqueue the FP32 throughput probe (dependent-FMA chains) on the context
    stream; returns (out buffer, FP32 operations of the launch)."""
    h = _h(ctx)
    if out is None:
        sms = torch.cuda.get_device_properties(device if device is not None else torch.cuda.current_device())
        out = torch.empty(8 * sms.multi_processor_count, dtype=torch.float32,
                          device=device if device is not None else "cuda")
    fl = C.c_double(0.0)
    N.check("mkf_fp32_probe", N.lib().mkf_fp32_probe(h, int(iters), _ptr(out), C.byref(fl)))
    return out, fl.value


def mkf_mlp_train_step(ctx, feat, label, w, m, v, t, w_bf16, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss=None):
    """One Adam step on the batch (w, m, v, w_bf16 updated in place)."""
    n = feat.shape[0]
    _need(feat, "feat", torch.float32, (n, N.MLP_IN))
    _need(label, "label", torch.float32, (n,))
    for name, t_ in (("w", w), ("m", m), ("v", v)):
        _need(t_, name, torch.float32, (N.MLP_PARAMS,))
    _need(w_bf16, "w_bf16", torch.int16, (N.MLP_PARAMS,))
    hp = N.MkfAdam(lr, beta1, beta2, eps)
    N.check("mkf_mlp_train_step", N.lib().mkf_mlp_train_step(
        _h(ctx), _ptr(feat), _ptr(label), n, _ptr(w), _ptr(m), _ptr(v), int(t), C.byref(hp), _ptr(w_bf16),
        _ptr(loss)))


class Context:
    """Convenience wrapper: one library context on one device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self.device = int(device)
        self.handle = mkf_create(self.device, stream)
        self.layers = None

    def close(self):
        if self.handle:
            mkf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        mkf_set_stream(self.handle, stream)

    def sync(self):
        mkf_sync(self.handle)

    def geometry_load(self, layers, bz, plans=None, region_eta_edges=None, field_alpha=None, material_map=None):
        mkf_geometry_load(self.handle, layers, bz, plans, region_eta_edges, field_alpha, material_map)
        self.layers = [dict(d) for d in layers]

    def geometry_field(self, kind, alpha=0.0):
        mkf_geometry_field(self.handle, kind, alpha)

    def hits_bin(self, xyz, layer, event_offsets, bins=None):
        return mkf_hits_bin(self.handle, xyz, layer, event_offsets, bins, self.device)

    def fit(self, xyz, hit_layer, hit_idx, seed_par=None, seed_cov=None, out=None):
        return mkf_fit(self.handle, xyz, hit_layer, hit_idx, seed_par, seed_cov, out, self.device)

    def seeds_clean(self, seed_hits, n_hits, seed_par, max_dqpt=0.5, max_deta=0.02, max_dphi=0.02, keep=None):
        return mkf_seeds_clean(self.handle, seed_hits, n_hits, seed_par, max_dqpt, max_deta, max_dphi, keep,
                               self.device)

    def tracks_dedup(self, hit_idx, n_hits, track_nhits, chi2, min_frac=0.5, keep=None):
        return mkf_tracks_dedup(self.handle, hit_idx, n_hits, track_nhits, chi2, min_frac, keep, self.device)

    def fit_backward(self, xyz, hit_layer, hit_idx, last_par, last_cov, inflate=100.0, out=None):
        return mkf_fit_backward(self.handle, xyz, hit_layer, hit_idx, last_par, last_cov, inflate, out, self.device)

    def fit_smooth(self, xyz, hit_layer, hit_idx, seed_par=None, seed_cov=None, inflate=100.0, out=None):
        return mkf_fit_smooth(self.handle, xyz, hit_layer, hit_idx, seed_par, seed_cov, inflate, out, self.device)

    def find(self, bins, seed_hits, seed_event, n_best=10, chi2_cut=30.0, max_consec_miss=3, max_out=None,
             out=None, counters=True, block_threads=0, mlp_bf16=None, mlp_tau=0.0, feat=None, event_times=None,
             seed_list=None, seed_count=None, mlp_mode=0, seed_order=0):
        nl = len(self.layers) if self.layers else None
        return mkf_find(self.handle, bins, seed_hits, seed_event, n_best, chi2_cut, max_consec_miss, max_out, nl, out,
                        counters, block_threads, self.device, mlp_bf16, mlp_tau, feat, event_times, seed_list,
                        seed_count, mlp_mode, seed_order)

    def seeds_where(self, status, bits, seed_list=None, seed_count=None):
        return mkf_seeds_where(self.handle, status, bits, seed_list, seed_count)
