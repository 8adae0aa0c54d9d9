"""The C ABI library builds for sm_103a, loads, and exports every entry
point include/mcl.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mcl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mcl_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("mcl_expand", "mcl_prune_select_recover", "mcl_inflate_normalize", "mcl_chaos",
                 "mcl_run", "mcl_create", "mcl_destroy", "mcl_components", "mcl_symbolic"):
        assert want in names


def test_library_builds_and_exports_every_symbol():
    from paper_2002_10083_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2002_10083_gb300 import mcl
    assert set(declared_functions()) <= set(mcl.SIGNATURES)


def test_version_string_without_gpu():
    from paper_2002_10083_gb300 import mcl
    lib = mcl.load()
    assert b"sm_103a" in lib.mcl_version()


def test_create_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2002_10083_gb300 import mcl
    lib = mcl.load()
    h = ctypes.c_void_p()
    st = lib.mcl_create(ctypes.byref(h), 0, mcl._ALLOC(0), mcl._FREE(0), None)
    assert st != 0 and not h.value


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2002_10083_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "mcl_oracle" not in txt, f
