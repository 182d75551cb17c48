"""The C-ABI library loads, exports every declared symbol, and rejects bad
arguments before touching the GPU (these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2104_13248_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bp_create", "bp_create_from_matrices", "bp_filter", "bp_backproject",
                     "fp_project", "bp_destroy", "bp_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.PROTOTYPES, f"{name} has no ctypes prototype"


def _geom(**kw):
    g = _lib.bp_geometry()
    g.sid, g.sdd, g.n_views = 1000.0, 1500.0, 8
    g.nu, g.nv, g.du, g.dv = 64, 48, 0.8, 0.8
    g.nx, g.ny, g.nz = 16, 16, 16
    g.sx = g.sy = g.sz = 1.0
    for k, v in kw.items():
        setattr(g, k, v)
    return g


@pytest.mark.parametrize("field,value", [
    ("sid", 0.0), ("sid", 2000.0), ("sdd", float("nan")), ("n_views", 0), ("nu", 1),
    ("nx", 0), ("du", -0.1), ("sz", 0.0), ("ox", float("inf")),
])
def test_create_rejects_bad_geometry(lib, field, value):
    g = _geom(**{field: value})
    h = ctypes.c_void_p()
    st = lib.bp_create(ctypes.byref(g), ctypes.byref(h))
    assert st == _lib.BP_ERR_INVALID_ARG
    assert h.value is None
    assert lib.bp_last_error(None)


def test_create_rejects_volume_behind_source(lib):
    g = _geom(sid=10.0, sdd=20.0, nx=64, ny=64, sx=1.0, sy=1.0)   # corners beyond the source
    h = ctypes.c_void_p()
    assert lib.bp_create(ctypes.byref(g), ctypes.byref(h)) == _lib.BP_ERR_INVALID_ARG
    assert b"behind" in lib.bp_last_error(None)


def test_null_arguments(lib):
    assert lib.bp_create(None, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.bp_filter(None, None, None, 0, 1, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.bp_backproject(None, None, 0, None, 1, 1.0, 0, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.fp_project(None, None, None, 1, 1.0, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.bp_get_matrices(None, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.bp_set_pipeline_depth(None, 4) == _lib.BP_ERR_INVALID_ARG
    assert lib.it_fill(None, 5, 1.0, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.it_ratio(None, None, None, -1, 0.0, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.it_residual(None, None, None, None, 3, 0.0, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.it_mlem_update(None, None, None, 2, 0.0, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.it_sart_update(None, None, None, 2, 1.0, 0, 0.0, None) == _lib.BP_ERR_INVALID_ARG
    assert lib.it_fill(None, 0, 1.0, None) == _lib.BP_OK   # empty: nothing to do, no launch
    lib.bp_destroy(None)   # NULL-safe


def test_matrices_rejected_when_depth_not_positive(lib):
    import numpy as np
    P = np.zeros((2, 12))
    P[:, 11] = -1.0   # w = -1 everywhere
    h = ctypes.c_void_p()
    st = lib.bp_create_from_matrices(P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2, 8, 8, 4, 4, 4,
                                     ctypes.byref(h))
    assert st == _lib.BP_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()
