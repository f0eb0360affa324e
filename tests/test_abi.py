"""The C-ABI library loads and exports every function include/vqnqs.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

import synthetic_inputs as si
from conftest import ROOT


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(vqnqs_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_11296_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vqnqs_create", "vqnqs_log_psi", "vqnqs_local_energy", "vqnqs_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2212_11296_gb300 import _lib
    bound = {name for name, _, _ in _lib.SIGNATURES}
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in bound, f"{name} has no ctypes signature"


def test_num_params_matches_generator_layout(lib):
    for args in [(16, 2, 32, 16), (100, 4, 128, 64), (256, 8, 256, 256), (400, 12, 384, 512)]:
        assert lib.vqnqs_num_params(*args) == si.num_params(*args)


def test_create_rejects_bad_shapes_without_touching_a_gpu(lib):
    h = ctypes.c_void_p()
    w = (ctypes.c_float * 4)()
    # heads not dividing d_model, d_model not a multiple of 32, K = 0, too many sites
    for args in [(4, 1, 1.0, 2, 32, 3, 16), (4, 1, 1.0, 2, 48, 4, 16), (4, 1, 1.0, 2, 32, 4, 0),
                 (24, 1, 1.0, 2, 32, 4, 16)]:
        assert lib.vqnqs_create(*args, ctypes.cast(w, ctypes.c_void_p), ctypes.byref(h)) == 1
        assert not h.value
