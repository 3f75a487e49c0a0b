"""ctypes binding of libmkf.so (the C ABI declared in include/mkf.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmkf.so")

MKF_OK = 0
MKF_ERR_ARG = -1
MKF_ERR_GEOMETRY = -2
MKF_ERR_CAPACITY = -3
MKF_ERR_CUDA = -4
MKF_ERR_DEVICE_CHECK = -5

ST_UNREACHABLE = 1
ST_BADSEED = 2
ST_NONFINITE = 4
ST_BADS = 8
ST_MISSSTOP = 16
ST_TRUNC = 32
ST_AMBIG = 64

MAX_LAYERS = 64
STATIC_MAX_HITS = 1 << 22
STATIC_MAX_BINS = 1 << 22
MAX_NBEST = 16

# Symbols declared in include/mkf.h (checked by the ABI test).
EXPORTS = ("mkf_create", "mkf_destroy", "mkf_set_stream", "mkf_sync", "mkf_status_string", "mkf_geometry_load",
           "mkf_hits_bin", "mkf_hitbins_free", "mkf_hitbins_info", "mkf_hitbins_export", "mkf_hits_bin_static", "mkf_geometry_material", "mkf_geometry_field", "mkf_geometry_material_map", "mkf_fit", "mkf_fit_backward", "mkf_fit_smooth", "mkf_seeds_clean", "mkf_tracks_dedup", "mkf_find", "mkf_mlp_to_bf16",
           "mkf_mlp_forward", "mkf_mlp_grad", "mkf_mlp_train_step", "mkf_fp32_probe", "mkf_seeds_where")


class MkfLayer(C.Structure):
    _fields_ = [("kind", C.c_int32), ("r_or_z", C.c_float), ("lo", C.c_float), ("hi", C.c_float),
                ("sigma_u", C.c_float), ("sigma_v", C.c_float), ("n_phi_bins", C.c_int32), ("n_zr_bins", C.c_int32)]


class MkfPlan(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("layer_ids", C.POINTER(C.c_int32))]


class MkfFindParams(C.Structure):
    _fields_ = [("n_best", C.c_int32), ("chi2_cut", C.c_float), ("max_consec_miss", C.c_int32),
                ("block_threads", C.c_int32), ("mlp_bf16", C.c_void_p), ("mlp_tau", C.c_float),
                ("feat_out", C.c_void_p), ("feat_ref", C.c_void_p), ("feat_count", C.c_void_p),
                ("feat_cap", C.c_int32), ("event_times", C.c_void_p), ("seed_list", C.c_void_p),
                ("seed_count", C.c_void_p), ("mlp_mode", C.c_int32), ("seed_order", C.c_int32)]


MLP_IN = 12
MLP_HIDDEN = 64
MLP_PARAMS = MLP_IN * MLP_HIDDEN + 2 * MLP_HIDDEN + 1


class MkfAdam(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class MkfError(RuntimeError):
    def __init__(self, fn, status, text):
        super().__init__(f"{fn} failed: {status} ({text})")
        self.status = status


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library; raises if libmkf.so is missing (build it first)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmkf.so not found at {LIB_PATH}: run paper_1811_04141_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, f32, u32 = C.c_void_p, C.c_int32, C.c_float, C.c_uint32
            L.mkf_create.argtypes = [C.POINTER(vp), i32, vp]
            L.mkf_create.restype = i32
            L.mkf_destroy.argtypes = [vp]
            L.mkf_destroy.restype = None
            L.mkf_set_stream.argtypes = [vp, vp]
            L.mkf_set_stream.restype = i32
            L.mkf_sync.argtypes = [vp]
            L.mkf_sync.restype = i32
            L.mkf_status_string.argtypes = [i32]
            L.mkf_status_string.restype = C.c_char_p
            L.mkf_geometry_load.argtypes = [vp, C.POINTER(MkfLayer), i32, C.POINTER(MkfPlan), i32,
                                            C.POINTER(f32), f32]
            L.mkf_geometry_load.restype = i32
            L.mkf_hits_bin.argtypes = [vp, vp, vp, vp, i32, i32, C.POINTER(vp)]
            L.mkf_hits_bin.restype = i32
            L.mkf_hitbins_free.argtypes = [vp]
            L.mkf_hitbins_free.restype = None
            L.mkf_hitbins_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_int64)]
            L.mkf_hitbins_info.restype = i32
            L.mkf_hitbins_export.argtypes = [vp, vp, vp, vp, vp]
            L.mkf_hitbins_export.restype = i32
            L.mkf_hits_bin_static.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp, vp]
            L.mkf_hits_bin_static.restype = i32
            L.mkf_mlp_to_bf16.argtypes = [vp, vp, vp, i32]
            L.mkf_mlp_to_bf16.restype = i32
            L.mkf_mlp_forward.argtypes = [vp, vp, vp, i32, vp]
            L.mkf_mlp_forward.restype = i32
            L.mkf_mlp_grad.argtypes = [vp, vp, vp, vp, i32, vp, vp]
            L.mkf_mlp_grad.restype = i32
            L.mkf_mlp_train_step.argtypes = [vp, vp, vp, i32, vp, vp, vp, i32, C.POINTER(MkfAdam), vp, vp]
            L.mkf_mlp_train_step.restype = i32
            L.mkf_fp32_probe.argtypes = [vp, i32, vp, C.POINTER(C.c_double)]
            L.mkf_fp32_probe.restype = i32
            L.mkf_seeds_where.argtypes = [vp, vp, i32, C.c_uint32, vp, vp]
            L.mkf_seeds_where.restype = i32
            L.mkf_fit.argtypes = [vp, vp, vp, i32, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp]
            L.mkf_fit.restype = i32
            L.mkf_fit_backward.argtypes = [vp, vp, vp, i32, vp, i32, i32, vp, vp, C.c_float, vp, vp, vp, vp, vp]
            L.mkf_fit_backward.restype = i32
            L.mkf_fit_smooth.argtypes = [vp, vp, vp, i32, vp, i32, i32, vp, vp, C.c_float, vp, vp, vp, vp, vp]
            L.mkf_fit_smooth.restype = i32
            L.mkf_geometry_material.argtypes = [vp, vp, vp, i32]
            L.mkf_geometry_material.restype = i32
            L.mkf_geometry_field.argtypes = [vp, i32, C.c_float]
            L.mkf_geometry_field.restype = i32
            L.mkf_geometry_material_map.argtypes = [vp, i32, i32, C.c_float, C.c_float, C.c_float, vp, vp]
            L.mkf_geometry_material_map.restype = i32
            L.mkf_seeds_clean.argtypes = [vp, vp, i32, i32, vp, C.c_float, C.c_float, C.c_float, vp]
            L.mkf_seeds_clean.restype = i32
            L.mkf_tracks_dedup.argtypes = [vp, vp, i32, i32, i32, vp, vp, C.c_float, vp]
            L.mkf_tracks_dedup.restype = i32
            L.mkf_find.argtypes = [vp, vp, vp, vp, i32, C.POINTER(MkfFindParams), vp, vp, vp, vp, vp, i32, vp, vp]
            L.mkf_find.restype = i32
            _lib = L
    return _lib


def check(fn: str, status: int) -> None:
    if status != MKF_OK:
        raise MkfError(fn, status, lib().mkf_status_string(status).decode())


def status_string(status: int) -> str:
    return lib().mkf_status_string(int(status)).decode()
