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


_STRUCTS = {"umgs_gaussians": "CGaussians", "umgs_mesh": "CMesh", "umgs_camera": "CCamera",
            "umgs_gaussian_grads": "CGaussianGrads", "umgs_mesh_grads": "CMeshGrads",
            "umgs_render_opts": "CRenderOpts", "umgs_frame_stats": "CFrameStats"}


def test_binding_structs_match_the_header(tmp_path):
    """Size and every field offset of the ctypes mirrors equal the C structs
    of include/umgs.h (compiled with the host C compiler)."""
    import shutil
    import subprocess
    from paper_2601_19233_gb300 import umgs
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "umgs.h"', "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in getattr(umgs, pyname)._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for cname, pyname in _STRUCTS.items():
        cls = getattr(umgs, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_default_render_opts(libpath):
    from paper_2601_19233_gb300 import umgs
    o = umgs.render_opts()
    assert (o.tile_size, o.blend_mode, o.flags, o.sched) == (16, umgs.BLEND_FULL, 0, 0)
    assert abs(o.t_eps - 1e-4) < 1e-9 and o.edge_sigma == 0.0
    s = umgs.render_opts(edge_sigma=0.5, save=True)
    assert s.flags == umgs.RENDER_SOFT_EDGE | umgs.RENDER_SAVE_BACKWARD and s.edge_sigma == 0.5
