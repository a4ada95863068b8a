"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/gm.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1302_5995_gb300 import build_ext
    return build_ext.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = declared_symbols()
    assert "gm_build" in names and "gm_solve" in names and "gm_free" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_the_same_symbols(lib_path):
    import paper_1302_5995_gb300 as gm
    assert set(gm.SIGNATURES) == set(declared_symbols())
    gm.load_library()


def test_strerror_and_free_null(lib_path):
    import paper_1302_5995_gb300 as gm
    lib = gm.load_library()
    assert gm.strerror(0) == "ok"
    assert "singular" in gm.strerror(gm.GM_ESINGULAR)
    lib.gm_free(None)  # NULL is a no-op


def test_missing_library_fails_loudly(tmp_path):
    import paper_1302_5995_gb300 as gm
    with pytest.raises(ImportError):
        gm._lib, saved = None, gm._lib
        try:
            gm.load_library(str(tmp_path / "nope.so"))
        finally:
            gm._lib = saved


def test_plan_tables_only_sm103a(lib_path):
    from paper_1302_5995_gb300 import build_ext
    assert build_ext.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
