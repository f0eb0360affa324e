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
