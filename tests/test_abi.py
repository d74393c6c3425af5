"""The C-ABI library builds, loads and exports every symbol include/geomhd.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "geomhd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(geo_[a-z0-9_A-Z]+)\s*\(", txt)))


def test_library_exports_header_symbols():
    from paper_1905_02504_gb300 import _build
    _build.build()
    lib = ctypes.CDLL(_build.LIB)
    syms = declared_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(lib, s), s
    from paper_1905_02504_gb300 import geomhd
    assert set(syms) <= set(geomhd.EXPORTED)


def test_errors_are_status_codes_without_gpu():
    from paper_1905_02504_gb300 import geomhd
    import pytest
    with pytest.raises(geomhd.GeoError):
        geomhd.geo_mesh_create(1, 2, 1.0, 2.0, 3)          # subdiv too small -> GEO_ERR_ARG
    with pytest.raises(geomhd.GeoError):
        geomhd.geo_mesh_create(4, 4, 2.0, 1.0, 3)          # r_out < r_in
    assert "r_in" in geomhd.geo_last_error()
