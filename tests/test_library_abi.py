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


def test_noalloc_refuses_sizes_beyond_its_array():
    # the allocation-free totals keep n_s * ceil(n_zone / 64) partials in a
    # fixed device array; a larger request is refused on the host with
    # BT_ERR_ARG before anything touches the device (the pointers are never
    # dereferenced)
    from paper_2003_02845_gb300 import build
    lib = ctypes.CDLL(build.build())
    fn = lib.bt_weighted_totals_noalloc
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    fn.argtypes = [vp, i32, i32, i32, i32, i32, vp, vp, vp, vp]
    fn.restype = i32
    limit = 1 << 16
    dummy = vp(16)
    for n_s, n_zone in ((2, 64 * limit), (1, 64 * limit + 1), (limit + 1, 1)):
        assert fn(dummy, 0, n_s, n_zone, 4, 8, dummy, dummy, dummy, None) == -1
    # sizes, precision and pointers are checked the same way
    assert fn(dummy, 0, 0, 1, 1, 1, dummy, dummy, dummy, None) == -1
    assert fn(dummy, 7, 1, 1, 1, 1, dummy, dummy, dummy, None) == -1
    assert fn(None, 0, 1, 1, 1, 1, dummy, dummy, dummy, None) == -1
