"""Ragged batch (several lattice sizes through one pipeline) through the C ABI.

Shared model: 6 layers, d_model 192, 6 heads, codebook 128, position
embeddings for up to 20 x 20 sites.  Lattices 6x6, 8x8, 12x12 and 20x20.
* bitwise equal to separate single-lattice calls whose weight blob holds the
  first L^2 position-embedding rows (rows are computed independently of the
  batch), in FP32 and BF16;
* FP32 E_loc within 1e-5 of the FP64 oracle on sampled outputs (near-tie rule of
  test_gpu_parity).
"""
import numpy as np
import pytest
import torch

import synthetic_inputs as si
from oracle import hamiltonian, model

pytestmark = pytest.mark.gpu
LAYERS, D, HEADS, K, LMAX = 6, 192, 6, 128, 20
GROUPS = [(6, 24), (8, 20), (12, 10), (20, 4)]


def sliced_blob(blob, L):
    """The blob for an L x L lattice: the first L^2 position-embedding rows."""
    nmax = LMAX * LMAX
    head = 3 * D
    return np.concatenate([blob[:head], blob[head:head + L * L * D], blob[head + nmax * D:]]).astype(np.float32)


@pytest.mark.parametrize("flags", [1, 3])
def test_ragged_equals_separate_lattices(flags):
    from paper_2212_11296_gb300 import VQNQS
    blob = si.make_weights(LMAX * LMAX, LAYERS, D, K, seed=0)
    big = VQNQS(LMAX, True, 1.0, LAYERS, D, HEADS, K, blob)
    groups = [(L, torch.as_tensor(si.make_samples(L, B, seed=1 + L)).cuda()) for L, B in GROUPS]
    e, mv = big.local_energy_ragged(groups, flags, want_mean_var=True)
    assert big.stats()["device_status"] == 0
    parts, off = [], 0
    for L, s in groups:
        small = VQNQS(L, True, 1.0, LAYERS, D, HEADS, K, sliced_blob(blob, L))
        ref = small.local_energy(s, flags)
        assert torch.equal(e[off:off + s.shape[0]], ref), L
        parts.append(ref)
        off += s.shape[0]
    allv = torch.cat(parts).double().cpu().numpy()
    m = mv.cpu().numpy()
    assert abs(m[0] - allv.mean()) < 1e-9 * max(1, abs(allv.mean())) and abs(m[1] - allv.var()) < 1e-7 * max(1, allv.var())


def test_ragged_fp32_against_oracle_sampled():
    from paper_2212_11296_gb300 import VQNQS
    blob = si.make_weights(LMAX * LMAX, LAYERS, D, K, seed=0)
    big = VQNQS(LMAX, True, 1.0, LAYERS, D, HEADS, K, blob)
    spins = {L: si.make_samples(L, B, seed=1 + L) for L, B in GROUPS}
    e = big.local_energy_ragged([(L, torch.as_tensor(spins[L]).cuda()) for L, _ in GROUPS], 1).cpu().numpy()
    off = 0
    for L, B in GROUPS:
        P = model.parse_blob(sliced_blob(blob, L), L * L, LAYERS, D, HEADS, K)
        pick = [0] if L == 20 else [0, B - 1]
        gap = np.empty(len(pick))
        want = hamiltonian.local_energy(P, spins[L][pick], L, True, 1.0, min_gap=gap)
        got = e[off + np.array(pick)]
        err = np.abs(got - want) / np.maximum(np.abs(want), 1e-3 * L * L)
        print(L, err, gap)
        assert np.all((err <= 1e-5) | (gap < 1e-6))
        off += B


def test_ragged_rejects_bad_groups():
    from paper_2212_11296_gb300 import VQNQS, VQNQSError
    big = VQNQS(8, True, 1.0, 1, 64, 2, 16, si.make_weights(64, 1, 64, 16))
    s = torch.as_tensor(si.make_samples(10, 2)).cuda()
    with pytest.raises(VQNQSError, match="ERR_ARG"):
        big.local_energy_ragged([(10, s)], 1)  # larger than the context's lattice
