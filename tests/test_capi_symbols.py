"""The C-ABI library builds, loads on a machine without a GPU, and exports every symbol
that include/gbri.h declares (no compute calls here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbri.h")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gbri_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_paths_calls():
    syms = declared_symbols()
    for name in ("phi", "phi_adjoint", "psi", "psi_adjoint", "prox_l1", "proj_l2ball", "solve"):
        assert "gbri_" + name in syms


def test_library_exports_every_declared_symbol():
    from paper_1903_04502_gb300 import _lib, build
    build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    # and the binding binds exactly the declared set
    assert set(_lib.SIGNATURES) == set(declared_symbols())


def test_binding_reports_version_and_errors_without_gpu():
    import paper_1903_04502_gb300 as g
    lib = g.library()
    assert lib.gbri_version().startswith(b"gbri")
    # argument validation happens before any CUDA call
    assert lib.gbri_plan_create(None, None, None, None) == -1
    assert b"null" in lib.gbri_last_error()


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    from paper_1903_04502_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _lib.load()
