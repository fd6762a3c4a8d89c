"""The C-ABI library loads on a machine without a GPU and exports every
function include/treepm_sr.h declares (no compute calls are made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "treepm_sr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1211_4406_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["tp_build_tree", "tp_short_range_force", "tp_short_range_vjp",
                     "tp_build_tree_batched", "tp_tree_free", "tp_tree_status"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1211_4406_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.tp_status_string.restype = ctypes.c_char_p
    assert lib.tp_status_string(0) == b"ok"
    assert lib.tp_status_string(-4) == b"capacity overflow"


def test_invalid_arguments_rejected_without_touching_the_gpu(lib):
    from paper_1211_4406_gb300 import _lib
    _lib.load()
    h = ctypes.c_void_p()
    p = _lib.params(r_cut=0.7)                                     # r_cut must be < 1/2
    assert _lib.load().tp_build_tree(None, None, 10, ctypes.byref(p), None, ctypes.byref(h)) == -1
    p = _lib.params(r_cut=0.1)
    assert _lib.load().tp_build_tree(None, None, -1, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert _lib.load().tp_tree_free(None) == 0


def test_pm_invalid_arguments_rejected_without_touching_the_gpu(lib):
    from paper_1211_4406_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    assert L.tp_pm_create(15, 0.2, 1.0, None, ctypes.byref(h)) == -1      # odd mesh
    assert L.tp_pm_create(4, 0.2, 1.0, None, ctypes.byref(h)) == -1       # below 8
    assert L.tp_pm_create(16, 0.5, 1.0, None, ctypes.byref(h)) == -1      # r_cut must be < 1/2
    assert L.tp_pm_create(16, 0.2, float("nan"), None, ctypes.byref(h)) == -1
    assert L.tp_pm_force(None, None, None, 10, None, 0, None) == -1
    assert L.tp_pm_vjp(None, None, None, 10, None, None, 0, None) == -1
    assert L.tp_pm_free(None) == 0


def test_stats_struct_layout_matches_the_header(tmp_path):
    """The binding's tp_stats mirrors the header's struct field by field: the
    same names in the same order at the same offsets (checked by compiling
    the header with the host C compiler)."""
    import subprocess

    from paper_1211_4406_gb300 import _lib
    fields = [f for f, _ in _lib.TPStats._fields_]
    assert "n_useful" in fields
    src = tmp_path / "layout.c"
    body = "".join(f'    printf("%s %zu\\n", "{f}", offsetof(tp_stats, {f}));\n' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "treepm_sr.h"\nint main(void) {\n'
                   f'{body}    printf("size %zu\\n", sizeof(tp_stats));\n    return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for f in fields:
        assert int(out[f]) == getattr(_lib.TPStats, f).offset, f
    assert int(out["size"]) == ctypes.sizeof(_lib.TPStats)
