"""The C-ABI library loads and exports every entry point that include/*.h
declares (no compute: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:int|size_t|void)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ut_decode", "ut_sort_hits", "compass_find", "compass_fit", "ut_ctx_create", "ut_status"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2002_11529_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2002_11529_gb300 as g
    monkeypatch.setattr(g._build, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(g, "_lib", None)
    with pytest.raises(RuntimeError):
        g.lib()


def test_workspace_size_is_host_only():
    import paper_2002_11529_gb300 as g
    g._lib = None
    assert g.decode_workspace_size(0) == 16
    assert g.decode_workspace_size(1000) == 16 + 8 * 1000
