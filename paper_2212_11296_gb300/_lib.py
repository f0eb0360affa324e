"""ctypes binding of libvqnqs.so (the C ABI in include/vqnqs.h).

Argument marshalling only: every step of the local-energy path runs in the
library's CUDA kernels.  Importing this module fails loudly when the library
has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvqnqs.so")

VQNQS_OK, VQNQS_ERR_ARG, VQNQS_ERR_CUDA, VQNQS_ERR_OOM, VQNQS_ERR_WORKSPACE, VQNQS_ERR_TIMEOUT, \
    VQNQS_ERR_INTERNAL = range(7)
REUSE = 1
BF16 = 2
INCREMENTAL = 4
BF16_SPLIT = 8
DEV_BAD_SPIN, DEV_HASH_OVERFLOW, DEV_TIMEOUT = 1, 2, 4
MAX_LAYERS = 64
NOALLOC_MAX_ROWS = 1 << 18

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_WORKSPACE", 5: "ERR_TIMEOUT",
                6: "ERR_INTERNAL"}


class Stats(ctypes.Structure):
    _fields_ = [
        ("samples", ctypes.c_int64),
        ("configs", ctypes.c_int64),
        ("rows", ctypes.c_int64),
        ("unique_rows", ctypes.c_int64 * (MAX_LAYERS + 1)),
        ("near_ties", ctypes.c_int64),
        ("flops_full", ctypes.c_double),
        ("flops_done", ctypes.c_double),
        ("device_status", ctypes.c_int32),
        ("active_rows", ctypes.c_int64),
        ("attn_pairs", ctypes.c_int64),
        ("inc_base_rows", ctypes.c_int64),
        ("inc_patched_rows", ctypes.c_int64),
        ("inc_certified_rows", ctypes.c_int64),
        ("inc_full_rows", ctypes.c_int64),
        ("inc_searched_rows", ctypes.c_int64),
        ("inc_patch_pairs", ctypes.c_int64),
        ("inc_full_pairs", ctypes.c_int64),
        ("inc_whole_pairs", ctypes.c_int64),
    ]


class StageTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("calls", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("ms", ctypes.c_double)]


MAX_STAGES = 32


class IncTuning(ctypes.Structure):
    _fields_ = [("patch_items", ctypes.c_int), ("rows_slices", ctypes.c_int), ("patch_ms", ctypes.c_float * 3),
                ("rows_ms", ctypes.c_float * 5)]


class Tuning(ctypes.Structure):
    _fields_ = [("qkv_bn", ctypes.c_int), ("mlp_up_bn", ctypes.c_int), ("mlp_down_bn", ctypes.c_int),
                ("ms", (ctypes.c_float * 4) * 3)]

# (name, restype, argtypes) of every exported symbol of include/vqnqs.h
SIGNATURES = [
    ("vqnqs_num_params", ctypes.c_size_t, [ctypes.c_int] * 4),
    ("vqnqs_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("vqnqs_create_tfim", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    ("vqnqs_create_arch", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("vqnqs_num_params_arch", ctypes.c_size_t, [ctypes.c_int] * 6),
    ("vqnqs_set_weights", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("vqnqs_sample_workspace_bytes", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("vqnqs_vmc_workspace_bytes", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("vqnqs_vmc_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_get_weights", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("vqnqs_sample", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_workspace_bytes", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("vqnqs_log_psi", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_local_energy_ragged", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 5 +
     [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_codes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3 +
     [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_local_energy", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_local_energy_codes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3 +
     [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_gemm_bf16", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_void_p]),
    ("vqnqs_gemm_bf16_split", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("vqnqs_grad_workspace_bytes", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("vqnqs_energy_grad_partials_workspace_bytes", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("vqnqs_energy_grad_partials", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3 +
     [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_energy_grad_combine", ctypes.c_int, [ctypes.c_void_p] * 5),
    ("vqnqs_grad_log_psi", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 5 +
     [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_vq_assign", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("vqnqs_compress_workspace_bytes", ctypes.c_size_t, [ctypes.c_int]),
    ("vqnqs_compress_rows", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 7 +
     [ctypes.c_size_t, ctypes.c_void_p]),
    ("vqnqs_autotune_chunk", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("vqnqs_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.POINTER(Tuning), ctypes.c_void_p]),
    ("vqnqs_autotune_incremental", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(IncTuning),
                                                  ctypes.c_void_p]),
    ("vqnqs_compress_rows_noalloc", ctypes.c_int, [ctypes.c_int] + [ctypes.c_void_p] * 7),
    ("vqnqs_check_timeout_path", ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]),
    ("vqnqs_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    ("vqnqs_reset_stats", ctypes.c_int, [ctypes.c_void_p]),
    ("vqnqs_profile_enable", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("vqnqs_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(StageTime), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
    ("vqnqs_launch_count", ctypes.c_int64, [ctypes.c_void_p]),
    ("vqnqs_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("vqnqs_destroy", None, [ctypes.c_void_p]),
]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libvqnqs.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
