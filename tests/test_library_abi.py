"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/bt.h (no device calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bt_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("bt_create", "bt_set_background", "bt_step", "bt_moments", "bt_totals", "bt_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2003_02845_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2003_02845_gb300 import bt, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bt, "_lib", None)
    with pytest.raises(RuntimeError):
        bt.lib()
