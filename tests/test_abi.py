"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/tmd.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "tmd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(tmd_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("tmd_create", "tmd_decode_frame", "tmd_submit", "tmd_poll", "tmd_destroy"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    from paper_2411_02206_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in declared_entry_points():
        assert hasattr(lib, n), f"{n} not exported"


def test_binding_uses_the_c_names():
    from paper_2411_02206_gb300 import tmd
    L = tmd.lib()
    for n in declared_entry_points():
        assert getattr(L, n).restype is not None


def test_product_path_does_not_import_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle|import\s+oracle)|liboracle|tmd_oracle", re.M)
    pkg = os.path.join(ROOT, "paper_2411_02206_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert not pat.search(open(os.path.join(dirpath, f)).read()), f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2411_02206_gb300 import tmd
    monkeypatch.setattr(tmd, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(tmd, "_lib", None)
    with pytest.raises(RuntimeError):
        tmd.lib()
