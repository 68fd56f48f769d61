"""The C-ABI library builds for sm_103a, loads, and exports every function
include/dvqls.h declares; the binding wraps each of them.  No compute call
is made (this file runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_].*?\b(dvqls_\w+)\s*\(", txt, re.M)
    return names


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_14435_gb300 import dvqls
    return dvqls


def test_every_declared_symbol_is_exported(built):
    lib = ctypes.CDLL(built.LIB_PATH)
    names = declared()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_function(built):
    for name in declared():
        assert name in built.EXPORTED, name
        assert callable(getattr(built, name)), name


def test_library_is_sm_103a_only(built):
    """The object files are built with one -gencode for sm_103a."""
    from paper_2604_14435_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2604_14435_gb300 import dvqls
    monkeypatch.setattr(dvqls, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(dvqls, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        dvqls.lib()


def test_create_without_gpu_is_an_error(built):
    """With no visible device dvqls_create returns a status, never crashes."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(built.DvqlsError):
        built.dvqls_create(0)
