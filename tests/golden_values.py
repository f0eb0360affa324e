"""Readers of the stored oracle values under tests/golden/ (written by the
scripts beside them, which call only oracle/)."""
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def eloc_16x16():
    """FP64 oracle values of the first 64 samples of the 16x16 workload
    (tests/golden/make_eloc_16x16.py): (e_loc, log_psi, min_relative_code_gap)."""
    rows = np.loadtxt(os.path.join(HERE, "eloc_16x16_64.txt"), comments="#")
    assert np.array_equal(rows[:, 0], np.arange(len(rows)))
    return rows[:, 1], rows[:, 2], rows[:, 3]


def check_fp32_against_golden(err, gap, tol=1e-5, flip_tol=1e-4, min_within=0.75):
    """FP32-path parity on stored samples: every sample within ``flip_tol``, at least
    ``min_within`` of them within ``tol``, and every sample beyond ``tol`` meets an
    oracle codeword near tie (relative gap < 1e-6) in one of its configurations,
    where FP32 and FP64 may pick different codewords (one such flip moves E_loc by
    up to ~1e-4 relative at 16x16)."""
    err, gap = np.asarray(err), np.asarray(gap)
    over = err > tol
    for i in np.argsort(-err)[:6]:
        print(f"sample {i}: rel err {err[i]:.3e}  oracle min gap {gap[i]:.3e}")
    assert err.max() <= flip_tol, f"largest relative error {err.max():.3e} > {flip_tol}"
    assert (~over).mean() >= min_within, f"{over.sum()} of {len(err)} samples beyond {tol}"
    assert not np.any(over & (gap >= 1e-6)), f"beyond {tol} without a near tie: {np.nonzero(over & (gap >= 1e-6))[0]}"


def eloc_variant(name):
    """Stored FP64 oracle values of a variant workload (tests/golden/make_eloc_variants.py):
    (e_loc, min_relative_code_gap) of its first 16 samples."""
    rows = np.loadtxt(os.path.join(HERE, f"eloc_{name}.txt"), comments="#")
    assert np.array_equal(rows[:, 0], np.arange(len(rows)))
    return rows[:, 1], rows[:, 2]
