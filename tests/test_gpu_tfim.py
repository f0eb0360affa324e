"""The transverse-field Ising chain (Sec. 4) through the C ABI against the FP64 oracle.

Same bars as the Heisenberg parity tests: FP32 E_loc within 1e-5 of the oracle
(denominator max(|E|, 1e-3 N)) on every sample whose oracle evaluation meets no
codeword near tie; BF16 within the BF16 path's distance.  Samples are chains
of independent uniform spins.
"""
import numpy as np
import pytest
import torch

import synthetic_inputs as si
from oracle import model, tfim

pytestmark = pytest.mark.gpu


def rel_err(got, want, N):
    return np.abs(np.asarray(got, np.float64) - want) / np.maximum(np.abs(want), 1e-3 * N)


def check(P, spins, got, periodic, J, G, tol=1e-5, max_miss=0.25):
    N = spins.shape[1]
    gap = np.empty(len(spins))
    want = tfim.local_energy(P, spins, periodic=periodic, J=J, Gamma=G, min_gap=gap)
    err = rel_err(got, want, N)
    miss = err > tol
    for i in np.argsort(-err)[:4]:
        print(f"sample {i}: rel err {err[i]:.3e}  min gap {gap[i]:.3e}")
    assert not np.any(miss & (gap >= 1e-6)), np.nonzero(miss & (gap >= 1e-6))[0]
    assert miss.mean() <= max_miss
    return want


def make(N, periodic, J, G, layers, d, heads, K, B, seed=1):
    from paper_2212_11296_gb300 import VQNQS
    w = si.make_weights(N, layers, d, K, seed=0)
    m = VQNQS.tfim_chain(N, periodic, J, G, layers, d, heads, K, w)
    P = model.parse_blob(w, N, layers, d, heads, K)
    spins = si.make_chain_samples(N, B, seed=seed)
    return m, P, spins, torch.as_tensor(spins).cuda()


@pytest.mark.parametrize("periodic,J,G", [(False, 1.0, 1.0), (True, 0.7, 1.3)])
def test_chain16_fp32_all_flags_match_oracle(periodic, J, G):
    from paper_2212_11296_gb300 import INCREMENTAL, REUSE
    m, P, spins, s = make(16, periodic, J, G, 2, 64, 2, 16, 64)
    e0 = m.local_energy(s, 0).cpu().numpy()
    check(P, spins, e0, periodic, J, G)
    e1 = m.local_energy(s, REUSE).cpu().numpy()
    assert np.array_equal(e0, e1)  # reuse == full recompute, bitwise
    e2 = m.local_energy(s, REUSE | INCREMENTAL).cpu().numpy()
    assert np.max(rel_err(e2, e1.astype(np.float64), 16)) <= 1e-5
    assert m.stats()["device_status"] == 0


def test_chain64_fp32_and_bf16():
    from paper_2212_11296_gb300 import BF16, INCREMENTAL, REUSE
    m, P, spins, s = make(64, False, 1.0, 1.0, 2, 128, 4, 32, 32)
    e = m.local_energy(s, REUSE).cpu().numpy()
    check(P, spins[:12], e[:12], False, 1.0, 1.0)
    ei = m.local_energy(s, REUSE | INCREMENTAL).cpu().numpy()
    assert (rel_err(ei, e.astype(np.float64), 64) > 1e-5).mean() <= 0.05
    eb = m.local_energy(s, REUSE | BF16 | INCREMENTAL).cpu().numpy()
    d = rel_err(eb, e.astype(np.float64), 64)
    print(f"BF16 incremental vs FP32 reuse: median {np.median(d):.2e} max {d.max():.2e}")
    assert np.median(d) <= 1e-2 and d.max() <= 0.1


def test_chain384_paper_size_sampled():
    """Sec. 4's largest chain: 384 sites, one block of width 256 with 8 heads."""
    from paper_2212_11296_gb300 import BF16, INCREMENTAL, REUSE
    from golden_values import check_fp32_against_golden, eloc_variant
    m, P, spins, s = make(384, False, 1.0, 1.0, 1, 256, 8, 64, 16)
    e = m.local_energy(s, REUSE).cpu().numpy()
    want, gap = eloc_variant("chain384")  # stored FP64 oracle values of these 16 chains
    check_fp32_against_golden(rel_err(e, want, 384), gap)
    eb = m.local_energy(s, REUSE | BF16 | INCREMENTAL).cpu().numpy()
    d = rel_err(eb, e.astype(np.float64), 384)
    print(f"384 sites, BF16 incremental vs FP32 reuse: median {np.median(d):.2e} max {d.max():.2e}")
    assert d.max() <= 0.1
    assert m.stats()["device_status"] == 0


def test_log_psi_same_as_on_a_lattice_context():
    """log psi depends on the weights and the spins only: a 16-site chain and a 4x4 lattice agree bitwise."""
    from paper_2212_11296_gb300 import VQNQS
    w = si.make_weights(16, 2, 64, 16, seed=0)
    chain = VQNQS.tfim_chain(16, False, 1.0, 1.0, 2, 64, 2, 16, w)
    lattice = VQNQS(4, True, 1.0, 2, 64, 2, 16, w)
    s = torch.as_tensor(si.make_chain_samples(16, 32, seed=5)).cuda()
    assert torch.equal(chain.log_psi(s), lattice.log_psi(s))


def test_ragged_rejects_a_chain_context():
    from paper_2212_11296_gb300 import VQNQS, VQNQSError
    m = VQNQS.tfim_chain(16, False, 1.0, 1.0, 1, 64, 2, 16, si.make_weights(16, 1, 64, 16))
    with pytest.raises(VQNQSError):
        m.local_energy_ragged([(4, torch.zeros(2, 16, dtype=torch.uint8, device="cuda"))])
