"""The C-ABI library loads and exports every symbol include/mkf.h declares (CPU only:
no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libmkf():
    from paper_1811_04141_gb300 import build
    build.build()
    from paper_1811_04141_gb300 import _native
    return _native.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mkf_[a-z0-9_]+)\s*\(", txt))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mkf_geometry_load", "mkf_hits_bin", "mkf_fit", "mkf_find"):
        assert required in names


def test_library_exports_every_declared_symbol(libmkf):
    for name in sorted(_declared()):
        assert hasattr(libmkf, name), name
    from paper_1811_04141_gb300 import _native
    assert set(_native.EXPORTS) == _declared()


def test_status_strings_and_errors_without_gpu(libmkf):
    from paper_1811_04141_gb300 import _native as N
    assert N.status_string(0) == "ok"
    assert "argument" in N.status_string(N.MKF_ERR_ARG)
    # NULL arguments are rejected before any CUDA call
    assert libmkf.mkf_create(None, 0, None) == N.MKF_ERR_ARG
    assert libmkf.mkf_sync(None) == N.MKF_ERR_ARG
    assert libmkf.mkf_fit(None, None, None, 0, None, 1, 0, None, None, None, None, None, None, None) == N.MKF_ERR_ARG
    assert libmkf.mkf_hitbins_info(None, None, None, None) == N.MKF_ERR_ARG
    assert libmkf.mkf_fit_smooth(None, None, None, 0, None, 1, 0, None, None, ctypes.c_float(100.0), None, None,
                                 None, None, None) == N.MKF_ERR_ARG
    assert libmkf.mkf_geometry_field(None, 1, ctypes.c_float(1e-5)) == N.MKF_ERR_ARG
    assert libmkf.mkf_geometry_material(None, None, None, 0) == N.MKF_ERR_ARG
    assert libmkf.mkf_geometry_material_map(None, 1, 1, ctypes.c_float(1.0), ctypes.c_float(0.0), ctypes.c_float(1.0),
                                            None, None) == N.MKF_ERR_ARG


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1811_04141_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"\bimport\s+oracle|from\s+oracle|liboracle", txt), fn
