"""Host-only checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/skim.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(skim_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("skim_create", "skim_build_sketches", "skim_greedy", "skim_oracle_query", "skim_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol():
    import ctypes

    from paper_1408_6282_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_and_argument_errors_without_gpu():
    import ctypes

    import paper_1408_6282_gb300 as pkg
    pkg.load()
    assert pkg.skim_strerror(0) == "ok"
    assert "invalid" in pkg.skim_strerror(-1)
    lib = pkg.load()
    # null arguments are rejected before any device call
    assert lib.skim_create(None, None, None, None) == -1
    assert lib.skim_build_sketches(None) == -1
    out = ctypes.c_void_p()
    g = pkg.skim_graph(0, 0, None, None, 0)
    p = pkg.skim_params(4, 4, 0, 0.1, 0, 0, 0, 0, 0)
    assert lib.skim_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(out)) == -1  # n == 0
    g = pkg.skim_graph(4, 0, None, None, 0)
    for bad in (pkg.skim_params(0, 4, 0, 0.1, 0, 0, 0, 0, 0), pkg.skim_params(65, 4, 0, 0.1, 0, 0, 0, 0, 0),
                pkg.skim_params(4, 1, 0, 0.1, 0, 0, 0, 0, 0), pkg.skim_params(4, 4, 0, 0.0, 0, 0, 0, 0, 0),
                pkg.skim_params(4, 4, 3, 0.1, 0, 0, 0, 0, 0), pkg.skim_params(4, 4, 0, 0.1, 0, 0, 0, 0, 3),
                pkg.skim_params(4, 4, 0, 0.1, 0, 0, 0, 0, 2)):  # bad rank mode; IC model needs l = 1
        assert lib.skim_create(ctypes.byref(g), ctypes.byref(bad), None, ctypes.byref(out)) == -1
    # entry points on a null context, checked before any device call
    buf = (ctypes.c_uint64 * 8)()
    ln = ctypes.c_uint32()
    assert lib.skim_get_sketch(None, 0, buf, ctypes.byref(ln)) == -1
    assert lib.skim_set_wait_limit_ns(None, 1000) == -1
    assert lib.skim_set_live_rows(None, 0) == -1
    t = pkg.skim_tuning(0, 8.0, 4)
    assert lib.skim_set_tuning(None, ctypes.byref(t)) == -1
    assert lib.skim_get_tuning(None, ctypes.byref(t)) == -1
    best = ctypes.c_uint32()
    assert lib.skim_autotune(None, ctypes.byref(t), 1, ctypes.byref(best), None) == -1
    # the allocation-free query rejects null pointers and unknown rank readings
    d = ctypes.c_double()
    assert lib.skim_union_estimate_static(None, None, 4, 4, 4, 0, None, 0, ctypes.byref(d), None) == -1
    assert lib.skim_union_estimate_static(buf, buf, 4, 4, 4, 3, None, 0, ctypes.byref(d), None) == -1
    assert lib.skim_union_estimate_static(buf, buf, 4, 4, 4, 2, None, 0, ctypes.byref(d), None) == -1  # IC: l = 1
    assert lib.skim_union_estimate_static(buf, buf, 4, 1, 4, 0, None, 0, ctypes.byref(d), None) == -1  # k < 2


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1408_6282_gb300 as pkg
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "libskim.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(RuntimeError, match="not found"):
        pkg.load()
