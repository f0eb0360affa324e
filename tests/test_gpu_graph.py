"""The local-energy path captured into one CUDA graph (uniform and ragged
batches) replays to the same bits as the eager calls, for new inputs too."""
import pytest
import torch

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("flags", [1, 3])
def test_uniform_graph_replay_equals_eager(flags):
    from paper_2212_11296_gb300 import LocalEnergyGraph, VQNQS
    L, layers, d, heads, K, B = 10, 4, 128, 8, 64, 96
    m = VQNQS(L, True, 1.0, layers, d, heads, K, si.make_weights(L * L, layers, d, K))
    g = LocalEnergyGraph(m, [(L, B)], flags)
    for seed in (1, 2):
        s = torch.as_tensor(si.make_samples(L, B, seed=seed)).cuda()
        got = g(s).clone()
        assert torch.equal(got, m.local_energy(s, flags))
    assert m.stats()["device_status"] == 0


def test_ragged_graph_replay_equals_eager():
    from paper_2212_11296_gb300 import LocalEnergyGraph, VQNQS
    layers, d, heads, K = 2, 192, 6, 128
    m = VQNQS(12, True, 1.0, layers, d, heads, K, si.make_weights(144, layers, d, K))
    shapes = [(6, 20), (8, 12), (12, 6)]
    g = LocalEnergyGraph(m, shapes, 3)
    for seed in (3, 4):
        spins = [torch.as_tensor(si.make_samples(L, B, seed=seed + L)).cuda() for L, B in shapes]
        got = g(*spins).clone()
        want = m.local_energy_ragged(list(zip([L for L, _ in shapes], spins)), 3)
        assert torch.equal(got, want)
