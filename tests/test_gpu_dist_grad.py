"""The sharded energy gradient through the C ABI on one GPU: the partial sums
of two halves of a batch (two ranks' shares), added as the all-reduce would,
then combined, against vqnqs_grad_log_psi's energy gradient of the whole batch
(Sec. 2 gradient estimator, seeds 2 (E - mean E) / B), and the FP64 mean and
variance against vqnqs_local_energy's.  The partials hold sum E O and sum O,
whose difference cancels about |mean E| / std E digits of the FP32 sums, so the
tolerance is 1e-4 of the largest gradient entry."""
import numpy as np
import pytest
import torch

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def test_halves_exchange_equals_whole_batch_gradient():
    from paper_2212_11296_gb300 import VQNQS
    from paper_2212_11296_gb300.dist import energy_gradient
    L, layers, d, heads, K, B = 4, 2, 32, 4, 16, 24
    N = L * L
    m = VQNQS(L, True, 1.0, layers, d, heads, K, si.make_weights(N, layers, d, K, seed=0))
    spins = torch.as_tensor(si.make_samples(L, B, seed=1)).cuda()
    e, mv = m.local_energy(spins, 0, want_mean_var=True)
    _, ref = m.grad_log_psi(spins, e_loc=e)
    # one process: the helper uses the local sums as they are
    g1, mv1 = energy_gradient(m, spins, e)
    # two ranks' shares, summed as the all-reduce sums them
    h = B // 3
    p = m.energy_grad_partials(spins[:h].contiguous(), e[:h].contiguous()) + \
        m.energy_grad_partials(spins[h:].contiguous(), e[h:].contiguous())
    g2, mv2 = m.energy_grad_combine(p)
    # a rank without samples contributes zeros
    z = m.energy_grad_partials(spins[:0].contiguous(), e[:0].contiguous())
    torch.cuda.synchronize()
    assert torch.count_nonzero(z) == 0
    scale = ref.abs().max().item()
    for g, mvx in ((g1, mv1), (g2, mv2)):
        err = (g - ref).abs().max().item() / scale
        print(f"max |grad - ref| / max |ref| = {err:.2e}")
        assert err <= 1e-4
        assert abs(mvx[0].item() - mv[0].item()) <= 1e-9 * abs(mv[0].item())
        assert abs(mvx[1].item() - mv[1].item()) <= 1e-6 * mv[1].item() + 1e-9
