"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point declared in include/rt103.h (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2311_18558_gb300 import build
    build.build()
    from paper_2311_18558_gb300 import _lib
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_mirrors_header():
    from paper_2311_18558_gb300 import _lib
    assert set(_lib.SIGNATURES) == _declared()


def test_version_and_no_device(lib):
    assert lib.rt_version().decode().startswith("rt103")
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.rt_create(0, None, ctypes.byref(h))
    assert st != 0 and not h.value


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2311_18558_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "librt103.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()
