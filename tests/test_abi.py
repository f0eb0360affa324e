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


def declared_prototypes():
    """{name: number of parameters} of every function include/vqnqs.h declares."""
    out = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(vqnqs_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
            params = m.group(2).strip()
            out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_arity_matches_header():
    from paper_2212_11296_gb300 import _lib
    protos = declared_prototypes()
    assert set(protos) == set(declared_functions())
    for name, _, args in _lib.SIGNATURES:
        assert name in protos, name
        assert len(args) == protos[name], f"{name}: header {protos[name]} parameters, binding {len(args)}"


def test_num_params_arch_matches_generator_layout(lib):
    for n, layers, d, K in [(16, 2, 32, 16), (64, 3, 128, 64), (256, 3, 256, 64)]:
        for half in (0, 1):
            for G in (1, 2, 4):
                assert lib.vqnqs_num_params_arch(n, layers, d, K, half, G) == \
                    si.num_params(n, layers, d, K, bool(half), G), (n, half, G)
    assert lib.vqnqs_num_params_arch(16, 2, 32, 16, 0, 3) == 0  # three spins per token: not supported
    assert lib.vqnqs_num_params_arch(18, 2, 32, 16, 0, 4) == 0  # sites not a multiple of the group


def test_create_arch_rejects_bad_variants_without_touching_a_gpu(lib):
    h = ctypes.c_void_p()
    w = (ctypes.c_float * 4)()
    # (L, layers, d, heads, K, vq_heads, half_block, token_group)
    for L, layers, d, heads, K, H, half, G in [
            (4, 2, 32, 4, 16, 3, 0, 1),    # d_model not a multiple of the quantizer heads
            (4, 1, 64, 2, 512, 8, 0, 1),   # 8 heads x 9 bits: three heads per 32-bit word, over two words
            (4, 2, 32, 4, 16, 1, 0, 3),    # three spins per token
            (3, 2, 32, 4, 16, 1, 0, 2),    # 9 sites: not a multiple of two
            (4, 2, 32, 4, 16, 9, 0, 1)]:   # more than 8 quantizer heads
        rc = lib.vqnqs_create_arch(L, 1, 1.0, layers, d, heads, K, H, half, G, ctypes.cast(w, ctypes.c_void_p),
                                   ctypes.byref(h))
        assert rc == 1 and not h.value, (L, d, K, H, G)


def test_struct_mirrors_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets: a C
    program built with the host compiler against include/vqnqs.h prints them."""
    import shutil
    import subprocess

    from paper_2212_11296_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    mirrors = {"vqnqs_stats": _lib.Stats, "vqnqs_stage_time": _lib.StageTime,
               "vqnqs_inc_tuning": _lib.IncTuning, "vqnqs_tuning": _lib.Tuning}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "vqnqs.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'    printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(c, f): int(v) for c, f, v in (ln.split() for ln in out if ln.strip())}
    for cname, py in mirrors.items():
        assert got[(cname, ".")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
