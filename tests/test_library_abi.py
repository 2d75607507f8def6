"""The C-ABI library builds, loads and exports every function include/vemsolve.h
declares (no compute: runs without a GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vemsolve.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(vem_[a-z_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1901_02330_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["vem_create", "vem_set_coefficient", "vem_set_source", "vem_assemble", "vem_solve",
              "vem_quadrature_points", "vem_last_error", "vem_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1901_02330_gb300 import vemsolve
    assert sorted(vemsolve._SIGS) == declared_functions()


def test_default_options_without_gpu(libpath):
    """vem_default_options is pure host code."""
    from paper_1901_02330_gb300 import vemsolve
    o = vemsolve.default_options()
    assert o.element == vemsolve.VEM_ELEMENT_E0 and o.restart == 30 and o.rtol == 1e-12
