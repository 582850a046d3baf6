"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads,
and exports every entry point that include/dmr.h declares; the product path
refuses to run without its library (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dmr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmr_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_all_declared_symbols():
    from paper_2202_11001_gb300.build import build_library

    path = build_library()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_declared_symbols():
    from paper_2202_11001_gb300 import dmr

    assert set(_declared()) <= set(dmr.exported_symbols())


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2202_11001_gb300 import dmr

    monkeypatch.setattr(dmr, "_lib", None)
    monkeypatch.setattr(dmr, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(dmr.DmrError):
        dmr.load()
