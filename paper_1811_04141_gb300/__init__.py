"""GB300-native (sm_103a) Kalman-filter track fitting and finding.

The compute path is libmkf.so (hand-written CUDA, C ABI in include/mkf.h);
`api` is its Python binding with the same names.  Build with `build.build()`.
"""
from .api import (Context, HitBins, mkf_create, mkf_destroy, mkf_find, mkf_fit, mkf_fit_backward, mkf_fit_smooth, mkf_geometry_field,
                  mkf_geometry_load, mkf_geometry_material, mkf_geometry_material_map,
                  mkf_hits_bin, mkf_seeds_clean, mkf_set_stream, mkf_sync, mkf_tracks_dedup)

__all__ = ["Context", "HitBins", "mkf_create", "mkf_destroy", "mkf_find", "mkf_fit", "mkf_fit_backward", "mkf_fit_smooth", "mkf_geometry_field",
           "mkf_geometry_load", "mkf_geometry_material", "mkf_geometry_material_map",
           "mkf_hits_bin", "mkf_seeds_clean", "mkf_set_stream", "mkf_sync", "mkf_tracks_dedup"]
