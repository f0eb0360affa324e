"""Pins of the oracle's codeword-gap diagnostic (oracle/model.py relative_gap and
segment_gap) against brute force.

The diagnostic decides which rows count as near ties of Eq. vq (relative gap
(l2 - l1) / l1 of the two smallest squared distances below 1e-6), so a wrong
second-best (top-2 over the wrong axis, a dropped square, the gap of the wrong
pair) would silently change which samples the parity tests exempt.  Here every
distance is summed directly, (o_t - w_t)^2 term by term in Python floats, and
the two smallest are picked by sorting.
"""
import math

import numpy as np
import torch

from oracle import model


def brute_gap(o_row, cb):
    d2 = sorted(sum((float(a) - float(b)) ** 2 for a, b in zip(o_row, w)) for w in cb)
    if len(d2) < 2:
        return math.inf
    return (d2[1] - d2[0]) / max(d2[0], 1e-30)


def test_relative_gap_matches_brute_force():
    rng = np.random.default_rng(5)
    o = rng.normal(size=(7, 3))
    cb = rng.normal(size=(5, 3))  # R != K so a top-2 over the wrong axis fails on shape or value
    got = model.relative_gap(torch.as_tensor(o), torch.as_tensor(cb)).numpy()
    want = np.array([brute_gap(o[r], cb) for r in range(7)])
    assert got.shape == (7,)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12)


def test_relative_gap_batched_rows_and_exact_tie():
    rng = np.random.default_rng(6)
    cb = rng.normal(size=(6, 4))
    o = rng.normal(size=(2, 3, 4))
    # row [1, 2] is the midpoint of codewords 2 and 4: their distances tie exactly,
    # and no other codeword is nearer (checked by brute force below)
    o[1, 2] = 0.5 * (cb[2] + cb[4])
    got = model.relative_gap(torch.as_tensor(o), torch.as_tensor(cb)).numpy()
    for i in range(2):
        for j in range(3):
            want = brute_gap(o[i, j], cb)
            assert abs(got[i, j] - want) <= 1e-9 * max(1.0, abs(want))
    d2 = [sum((a - b) ** 2 for a, b in zip(o[1, 2], w)) for w in cb]
    if min(d2) == d2[2]:
        assert abs(got[1, 2]) < 1e-12


def test_relative_gap_one_codeword_is_infinite():
    o = torch.randn(4, 3, dtype=torch.float64)
    cb = torch.randn(1, 3, dtype=torch.float64)
    assert torch.isinf(model.relative_gap(o, cb)).all()


def test_segment_gap_is_min_over_heads():
    rng = np.random.default_rng(7)
    H, K, dq = 3, 5, 2
    cb = rng.normal(size=(H, K, dq))
    o = rng.normal(size=(6, H * dq))
    got = model.segment_gap(torch.as_tensor(o), torch.as_tensor(cb)).numpy()
    want = np.array([min(brute_gap(o[r, h * dq:(h + 1) * dq], cb[h]) for h in range(H)) for r in range(6)])
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12)
    # one head: the same as relative_gap
    cb1 = rng.normal(size=(K, H * dq))
    np.testing.assert_allclose(model.segment_gap(torch.as_tensor(o), torch.as_tensor(cb1)).numpy(),
                               [brute_gap(o[r], cb1) for r in range(6)], rtol=1e-9, atol=1e-12)
