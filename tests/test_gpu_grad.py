"""Hand-written backward (vqnqs_grad_log_psi) against the FP64 oracle's
straight-through autograd (Sec. 3.1 Eq. st) and the energy-gradient assembly
(Sec. 2).  The GPU backward computes in FP32: entries must match to 2e-4 of the
largest |entry| of the same sample (FP32 sums over up to N * 4d terms)."""
import numpy as np
import pytest
import torch

import synthetic_inputs as si
from oracle import gradient, hamiltonian, model

pytestmark = pytest.mark.gpu
GRAD_TOL = 2e-4


def close(got, want, tol=GRAD_TOL):
    got = np.asarray(got, np.float64)
    scale = np.abs(want).max(axis=-1, keepdims=True)
    err = (np.abs(got - want) / scale).max()
    print(f"max |diff| / max|O| = {err:.3e}")
    return err <= tol


def setup(L, layers, d, heads, K, B, seed_w=0, std=0.02):
    from paper_2212_11296_gb300 import VQNQS
    N = L * L
    w = si.make_weights(N, layers, d, K, seed=seed_w, std=std)
    spins = si.make_samples(L, B, seed=1)
    return VQNQS(L, True, 1.0, layers, d, heads, K, w), model.parse_blob(w, N, layers, d, heads, K), spins


@pytest.mark.parametrize("std", [0.02, 0.3])
def test_per_sample_O_matches_oracle_4x4(std):
    m, P, spins = setup(4, 2, 32, 4, 16, 8, std=std)
    s = torch.as_tensor(spins).cuda()
    O, grad = m.grad_log_psi(s, want_O=True, want_grad=True)
    want = gradient.per_sample_O(P, spins)
    assert close(O.cpu().numpy(), want)
    assert close(grad.cpu().numpy()[None], want.sum(0)[None])
    assert m.stats()["device_status"] == 0


def test_energy_gradient_matches_oracle_4x4():
    m, P, spins = setup(4, 2, 32, 4, 16, 16, std=0.3)
    s = torch.as_tensor(spins).cuda()
    e = m.local_energy(s, 0)
    _, g = m.grad_log_psi(s, e_loc=e)
    e_ora = hamiltonian.local_energy(P, spins, 4, True, 1.0)
    want = gradient.energy_gradient(gradient.per_sample_O(P, spins), e_ora)
    assert close(g.cpu().numpy()[None], want[None], 1e-3)
    # the per-sample path and the folded-seed path agree
    O, g2 = m.grad_log_psi(s, e_loc=e, want_O=True)
    assert close(g2.cpu().numpy()[None], g.cpu().numpy()[None].astype(np.float64), 1e-5)


def test_chunked_gradient_equals_single_chunk():
    m, P, spins = setup(4, 2, 32, 4, 16, 16, std=0.3)
    s = torch.as_tensor(spins).cuda()
    seeds = torch.linspace(-1, 1, 16, device="cuda")
    _, g1 = m.grad_log_psi(s, seeds=seeds)
    _, g2 = m.grad_log_psi(s, seeds=seeds, chunk_samples=3)
    assert torch.allclose(g1, g2, rtol=1e-5, atol=1e-6 * g1.abs().max().item())


def test_autograd_function_matches_seeded_gradient():
    from paper_2212_11296_gb300 import LogPsi
    m, P, spins = setup(4, 2, 32, 4, 16, 8, std=0.3)
    s = torch.as_tensor(spins).cuda()
    w = torch.as_tensor(si.make_weights(16, 2, 32, 16, seed=0, std=0.3)).cuda().requires_grad_(True)
    lp = LogPsi.apply(w, s, m, 0)
    c = torch.arange(8, device="cuda", dtype=torch.float32) - 3.5
    (lp * c).sum().backward()
    _, g = m.grad_log_psi(s, seeds=c)
    assert torch.equal(w.grad, g)
    want = gradient.per_sample_O(P, spins).T @ c.cpu().numpy().astype(np.float64)
    assert close(w.grad.cpu().numpy()[None], want[None])


def test_differentiation_config_20x20_sampled():
    """20x20, 12 layers, d 384, 12 heads, K 512: O_k of 2 samples vs the oracle."""
    m, P, spins = setup(20, 12, 384, 12, 512, 2)
    s = torch.as_tensor(spins).cuda()
    O, _ = m.grad_log_psi(s, want_O=True, want_grad=False)
    want = gradient.per_sample_O(P, spins)
    assert close(O.cpu().numpy(), want, 1e-3)


def test_tensor_core_energy_gradient_matches_oracle_and_fp32():
    """VQNQS_BF16: the summed gradient's GEMMs (recomputed forward, dX = dY W^T,
    dW = X^T dY) on the tensor cores with split operands, d_model 64 and K 64:
    the energy gradient against the oracle's (1e-3 of its largest entry, as the
    FP32 backward) and against the FP32 backward (1e-4)."""
    from paper_2212_11296_gb300 import BF16
    m, P, spins = setup(4, 2, 64, 2, 64, 16, std=0.3)
    s = torch.as_tensor(spins).cuda()
    e = m.local_energy(s, 0)
    _, g_tc = m.grad_log_psi(s, e_loc=e, flags=BF16)
    _, g32 = m.grad_log_psi(s, e_loc=e)
    e_ora = hamiltonian.local_energy(P, spins, 4, True, 1.0)
    want = gradient.energy_gradient(gradient.per_sample_O(P, spins), e_ora)
    assert close(g_tc.cpu().numpy()[None], want[None], 1e-3)
    assert close(g_tc.cpu().numpy()[None], g32.cpu().numpy()[None].astype(np.float64), 1e-4)
    # seeded sums too (the weight-gradient GEMMs accumulate over rows)
    seeds = torch.linspace(-1, 1, 16, device="cuda")
    _, a = m.grad_log_psi(s, seeds=seeds, flags=BF16)
    _, b = m.grad_log_psi(s, seeds=seeds)
    assert close(a.cpu().numpy()[None], b.cpu().numpy()[None].astype(np.float64), 1e-4)
    assert m.stats()["device_status"] == 0


def test_tensor_core_gradient_differentiation_config_against_fp32():
    """20x20, 12 layers, d 384, 12 heads, K 512, 2 samples: the tensor-core
    gradient against the FP32 backward (1e-4 of the largest entry)."""
    from paper_2212_11296_gb300 import BF16
    m, P, spins = setup(20, 12, 384, 12, 512, 2)
    s = torch.as_tensor(spins).cuda()
    seeds = torch.tensor([1.0, -0.5], device="cuda")
    _, a = m.grad_log_psi(s, seeds=seeds, flags=BF16)
    _, b = m.grad_log_psi(s, seeds=seeds)
    assert close(a.cpu().numpy()[None], b.cpu().numpy()[None].astype(np.float64), 1e-4)
