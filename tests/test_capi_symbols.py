"""The C-ABI library builds, loads without a GPU and exports every function
that include/lb.h declares; the Python binding carries the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lb_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_0707_1299_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "lb_step" in names and "lb_create" in names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_has_the_c_names(lib):
    from paper_0707_1299_gb300 import lb
    lb.load()
    for n in _declared():
        assert callable(getattr(lb, n)), n
    assert set(lb.EXPORTS) == _declared()


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_0707_1299_gb300 import lb
    monkeypatch.setattr(lb, "_lib", None)
    monkeypatch.setattr(lb, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        lb.load()


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_0707_1299_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, flags=re.M), f
                assert "lb_oracle" not in src, f
