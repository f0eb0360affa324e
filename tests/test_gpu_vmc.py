"""One full variational Monte Carlo step (vqnqs_vmc_step, Sec. 2) against the oracle.

Sampling with the caller's uniforms (the oracle sampler's draws, near-tie rule
of test_gpu_sample), local energies of the drawn configurations (1e-5 of the
FP64 oracle), the energy gradient 2 mean[(E - mean E) O_k] against the oracle's
straight-through autograd (1e-3 of the largest entry, as test_gpu_grad), and the
update theta - lr * grad applied to the context's weights (exactly, in FP32),
with the derived tables rebuilt (the next evaluation uses the new weights).
"""
import numpy as np
import pytest
import torch

import synthetic_inputs as si
from oracle import gradient, hamiltonian, model, sampler

pytestmark = pytest.mark.gpu


def test_vmc_step_matches_oracle_4x4():
    from paper_2212_11296_gb300 import VQNQS
    L, layers, d, heads, K, B, lr = 4, 2, 32, 4, 16, 64, 0.05
    N = L * L
    w = si.make_weights(N, layers, d, K, seed=0, std=0.1)
    m = VQNQS(L, True, 1.0, layers, d, heads, K, w)
    P = model.parse_blob(w, N, layers, d, heads, K)
    u = si.uniforms(21, B * N).reshape(B, N).astype(np.float32)
    out = m.vmc_step(torch.as_tensor(u).cuda(), lr)
    spins = out["spins"].cpu().numpy()
    # the draws
    want, pup = sampler.sample(P, u.astype(np.float64))
    for b in np.nonzero(~np.all(spins == want, axis=1))[0]:
        p = int(np.argmax(spins[b] != want[b]))
        assert abs(float(u[b, p]) - pup[b, p]) < 1e-5
    # energies of the drawn configurations
    e = out["e_loc"].cpu().numpy()
    e_or = hamiltonian.local_energy(P, spins, L, True, 1.0)
    assert np.max(np.abs(e - e_or) / np.maximum(np.abs(e_or), 1e-3 * N)) <= 1e-5
    mv = out["mean_var"].cpu().numpy()
    e64 = e.astype(np.float64)
    assert abs(mv[0] - e64.mean()) <= 1e-12 * max(1.0, abs(e64.mean()))
    assert abs(mv[1] - e64.var()) <= 1e-9 * max(1.0, e64.var())
    # the gradient
    g = out["grad"].cpu().numpy().astype(np.float64)
    g_or = gradient.energy_gradient(gradient.per_sample_O(P, spins), e_or)
    err = np.max(np.abs(g - g_or)) / np.max(np.abs(g_or))
    print(f"gradient: max |diff| / max |grad| = {err:.3e}")
    assert err <= 1e-3
    # the update, applied in FP32
    w_new = m.weights().cpu().numpy()
    assert np.array_equal(w_new, (w - np.float32(lr) * out["grad"].cpu().numpy()).astype(np.float32))
    # the derived tables follow the new weights: log psi equals a fresh context's
    fresh = VQNQS(L, True, 1.0, layers, d, heads, K, w_new)
    s = torch.as_tensor(spins).cuda()
    assert torch.equal(m.log_psi(s), fresh.log_psi(s))
    assert not torch.equal(m.log_psi(s), VQNQS(L, True, 1.0, layers, d, heads, K, w).log_psi(s))
