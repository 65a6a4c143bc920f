"""The C-ABI library builds, loads and exports every symbol include/umgs.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(umgs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2601_19233_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("umgs_ctx_create", "umgs_render", "umgs_frame_lists"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2601_19233_gb300 import umgs
    monkeypatch.setattr(umgs, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(umgs, "_lib", None)
    with pytest.raises(RuntimeError):
        umgs.lib()


def test_ctx_create_rejects_bad_device(libpath):
    from paper_2601_19233_gb300 import umgs
    L = umgs.lib()
    h = ctypes.c_void_p()
    assert L.umgs_ctx_create(ctypes.byref(h), 12345) != 0
