"""Host-side checks of the C ABI (no GPU work): the library builds, loads and
exports every entry point include/msm.h declares; configuration validation
and workspace sizing run on the host."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(md_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libmsm():
    from paper_2205_14121_gb300 import build as B
    B.build()
    import paper_2205_14121_gb300 as M
    return M.lib()


def test_every_declared_symbol_is_exported(libmsm):
    names = declared_functions()
    assert "md_init" in names and "md_mts_step" in names
    for name in names:
        assert hasattr(libmsm, name), name


def test_workspace_size_and_validation(libmsm):
    import paper_2205_14121_gb300._binding as B
    cfg = B.config_for(24000, (20.0, 20.0, 20.0))
    nb = C.c_size_t()
    assert libmsm.md_workspace_size(C.byref(cfg), C.byref(nb)) == 0
    assert nb.value > 24000 * 200
    bad = B.config_for(100, (20.0, 20.0, 20.0), dt=-0.01)
    assert libmsm.md_workspace_size(C.byref(bad), C.byref(nb)) == -1
    bad = B.config_for(0, (20.0, 20.0, 20.0))
    assert libmsm.md_workspace_size(C.byref(bad), C.byref(nb)) == -1
    walls_le = B.config_for(24000, (20.0, 20.0, 20.0), walls=True)
    walls_le.flags |= B.MD_CFG_LEES_EDWARDS
    assert libmsm.md_workspace_size(C.byref(walls_le), C.byref(nb)) == -1


def test_init_rejects_small_workspace(libmsm):
    import paper_2205_14121_gb300._binding as B
    cfg = B.config_for(24000, (20.0, 20.0, 20.0))
    bufs = B.md_buffers(None, 0)
    h = C.c_void_p()
    assert libmsm.md_init(C.byref(cfg), C.byref(bufs), None, C.byref(h)) == -2
    assert b"workspace" in libmsm.md_last_error(None)


def test_product_path_has_no_oracle_import():
    """The engine package never reaches the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2205_14121_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "msm_oracle" not in text, fn
