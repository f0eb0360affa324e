"""The GEMM tile-width autotuner: it reports timings for every valid width,
keeps widths that divide each step's output width, and the path's results do
not change with the chosen widths (a row's K-reduction order is the same)."""
import pytest
import torch

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def test_autotune_choices_valid_and_results_unchanged():
    from paper_2212_11296_gb300 import BF16, REUSE, VQNQS
    L, layers, d, heads, K, B = 8, 2, 192, 6, 128, 64
    m = VQNQS(L, True, 1.0, layers, d, heads, K, si.make_weights(L * L, layers, d, K))
    s = torch.as_tensor(si.make_samples(L, B)).cuda()
    before = m.local_energy(s, REUSE | BF16).clone()
    t = m.autotune(M=4096)
    for bn, n in ((t["qkv_bn"], 3 * d), (t["mlp_up_bn"], 4 * d), (t["mlp_down_bn"], d)):
        assert bn in (64, 128, 192, 256) and n % bn == 0
    for step, n in enumerate((3 * d, 4 * d, d)):
        for i, w in enumerate((64, 128, 192, 256)):
            assert (t["ms"][step][i] > 0) == (n % w == 0)
    after = m.local_energy(s, REUSE | BF16)
    assert torch.allclose(after, before, rtol=1e-6, atol=0)
    assert m.stats()["device_status"] == 0
