"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/geneo.h declares (no GPU needed, no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "geneo.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(geneo_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_18783_gb300 import build as b
    path = b.LIB
    if not os.path.exists(path):
        b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["geneo_setup", "geneo_apply_preconditioner", "geneo_solve",
                     "geneo_destroy", "geneo_assemble_rhs"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_names_match(lib):
    import paper_2311_18783_gb300.api as api
    api.load_library()
    assert set(api._SIGS) == set(declared_functions())


def test_status_text_without_gpu(lib):
    lib.geneo_strerror.restype = ctypes.c_char_p
    assert lib.geneo_strerror(0) == b"ok"
    assert lib.geneo_strerror(-4) == b"matrix not positive definite"
