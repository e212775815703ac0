"""The C-ABI library loads and exports every function include/bddc_so.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bddc_so.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2001_07289_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    return ctypes.CDLL(build_lib.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("bddc_setup", "bddc_apply", "pcg_solve", "bddc_operator", "bddc_gradient", "bddc_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    pytest.importorskip("torch")
    from paper_2001_07289_gb300 import bddc
    assert set(bddc.EXPORTS) == set(declared_functions())


def test_null_arguments_rejected_without_gpu_work(lib):
    lib.bddc_setup.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.bddc_setup(None, None, None, None, None, ctypes.byref(out)) == -1
    assert lib.bddc_destroy(None) == 0
    lib.bddc_apply.restype = ctypes.c_int
    assert lib.bddc_apply(None, None, None, None) == -1
