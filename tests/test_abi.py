"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/*.h; the binding declares the same names."""
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
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*(dvm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1503_04544_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1503_04544_gb300 import dvm
    assert sorted(dvm.SIGNATURES) == _declared()


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1503_04544_gb300 import dvm
    monkeypatch.setattr(dvm, "_lib", None)
    monkeypatch.setattr(dvm, "LIB_PATH", str(tmp_path / "missing" / "libdvm.so"))
    import paper_1503_04544_gb300.build as b
    monkeypatch.setattr(b, "build", lambda *a, **k: (_ for _ in ()).throw(RuntimeError("no nvcc")))
    with pytest.raises(Exception):
        dvm.load()
