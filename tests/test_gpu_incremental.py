"""The incremental local-energy path (VQNQS_INCREMENTAL) through the C ABI.

A connected configuration's attention rows whose query equals the sample's are
corrected for the changed keys only (softmax identity), and their codeword is
taken from the sample's row only when a distance bound proves it unchanged;
everything else is recomputed.  The result is exact up to rounding, so the FP32
bars of the reuse path apply unchanged:
* E_loc within 1e-5 of the FP64 oracle except for samples whose oracle meets a
  codeword near tie (the rule of test_gpu_parity);
* E_loc within 1e-5 of the FP32 reuse path, except where the two FP32 paths
  round a codeword near tie differently (a few samples at most);
* the row counts partition: every row at or after a configuration's first
  changed site is a sample's own row, a patched row or a recomputed one.
BF16: E_loc within the BF16 path's own distance from the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import synthetic_inputs as si
from oracle import model
from test_gpu_parity import check_against_oracle, rel_err

pytestmark = pytest.mark.gpu

# name: (L, layers, d_model, heads, K, B); head widths 32 and 16
CONFIGS = {
    "4x4": (4, 2, 64, 2, 16, 64),
    "6x6": (6, 3, 64, 4, 32, 96),
    "10x10": (10, 4, 128, 8, 64, 512),
    "16x16": (16, 8, 256, 8, 256, 64),
}
_cache = {}


def setup(name, periodic=True, J=1.0):
    key = (name, periodic, J)
    if key not in _cache:
        from paper_2212_11296_gb300 import VQNQS
        L, layers, d, heads, K, B = CONFIGS[name]
        N = L * L
        w = si.make_weights(N, layers, d, K, seed=0)
        spins = si.make_samples(L, B, seed=1)
        m = VQNQS(L, periodic, J, layers, d, heads, K, w)
        P = model.parse_blob(w, N, layers, d, heads, K)
        _cache[key] = (m, P, spins, torch.as_tensor(spins).cuda())
    return _cache[key]


def check_partition(m, B, N, layers):
    s = m.stats()
    assert s["device_status"] == 0
    assert s["inc_base_rows"] == B * N * layers
    assert s["active_rows"] * layers == s["inc_base_rows"] + s["inc_patched_rows"] + s["inc_full_rows"]
    assert s["inc_searched_rows"] == s["inc_full_rows"] + s["inc_patched_rows"] - s["inc_certified_rows"]
    assert 0 <= s["inc_certified_rows"] <= s["inc_patched_rows"]
    return s


@pytest.mark.parametrize("name,periodic,J", [("4x4", True, 1.0), ("6x6", False, 0.7), ("6x6", True, 1.0)])
def test_fp32_matches_oracle(name, periodic, J):
    from paper_2212_11296_gb300 import INCREMENTAL, REUSE
    m, P, spins, s_dev = setup(name, periodic, J)
    L, layers = CONFIGS[name][0], CONFIGS[name][1]
    m.reset_stats()
    e = m.local_energy(s_dev, REUSE | INCREMENTAL).cpu().numpy()
    s = check_partition(m, len(spins), L * L, layers)
    check_against_oracle(P, spins, e, L, periodic, J, 1e-5)
    e_reuse = m.local_energy(s_dev, REUSE).cpu().numpy()
    assert np.max(rel_err(e, e_reuse.astype(np.float64), L * L, J)) <= 1e-5
    print(f"{name}: patched {s['inc_patched_rows']}, certified {s['inc_certified_rows']}, "
          f"recomputed {s['inc_full_rows']}, searched {s['inc_searched_rows']}")


def test_10x10_fp32_matches_reuse_path_and_sampled_oracle():
    from paper_2212_11296_gb300 import INCREMENTAL, REUSE
    m, P, spins, s_dev = setup("10x10")
    m.reset_stats()
    e = m.local_energy(s_dev, REUSE | INCREMENTAL).cpu().numpy()
    s = check_partition(m, len(spins), 100, 4)
    e_reuse = m.local_energy(s_dev, REUSE).cpu().numpy()
    err = rel_err(e, e_reuse.astype(np.float64), 100)
    print("largest differences vs reuse path:", np.sort(err)[-5:])
    assert (err > 1e-5).mean() <= 0.02
    assert s["inc_certified_rows"] > 0.5 * s["inc_patched_rows"]
    check_against_oracle(P, spins[:8], e[:8], 10, True, 1.0, 1e-5)


def test_16x16_fp32_and_bf16():
    from paper_2212_11296_gb300 import BF16, INCREMENTAL, REUSE
    m, P, spins, s_dev = setup("16x16")
    m.reset_stats()
    e = m.local_energy(s_dev, REUSE | INCREMENTAL).cpu().numpy()
    s = check_partition(m, len(spins), 256, 8)
    e_reuse = m.local_energy(s_dev, REUSE).cpu().numpy()
    err = rel_err(e, e_reuse.astype(np.float64), 256)
    print("FP32 incremental vs reuse, largest:", np.sort(err)[-5:])
    assert (err > 1e-5).mean() <= 0.05
    print(f"16x16: searched {s['inc_searched_rows']} of {s['active_rows'] * 8} active rows")
    assert s["inc_searched_rows"] < 0.5 * s["active_rows"] * 8
    from golden_values import check_fp32_against_golden, eloc_16x16
    want, _, gap = eloc_16x16()
    check_fp32_against_golden(rel_err(e[:len(want)], want, 256), gap)
    # BF16: the incremental path stays as close to the oracle as the BF16 reuse path
    m.reset_stats()
    eb = m.local_energy(s_dev, REUSE | BF16 | INCREMENTAL).cpu().numpy()
    check_partition(m, len(spins), 256, 8)
    eb_reuse = m.local_energy(s_dev, REUSE | BF16).cpu().numpy()
    d_inc = rel_err(eb, e_reuse.astype(np.float64), 256)
    d_reuse = rel_err(eb_reuse, e_reuse.astype(np.float64), 256)
    print(f"BF16 vs FP32 reuse: incremental median {np.median(d_inc):.2e} max {d_inc.max():.2e}; "
          f"reuse median {np.median(d_reuse):.2e} max {d_reuse.max():.2e}")
    assert np.median(d_inc) <= 2 * np.median(d_reuse) + 1e-4
    assert d_inc.max() <= 0.1


def test_bf16_four_heads_close_to_reuse_and_deterministic():
    """d_model 128 with 4 heads of 32: the BF16 path patches rows on the tensor
    cores in one four-head round."""
    from paper_2212_11296_gb300 import BF16, INCREMENTAL, REUSE, VQNQS
    L, layers, d, heads, K = 8, 3, 128, 4, 64
    w = si.make_weights(L * L, layers, d, K, seed=0)
    m = VQNQS(L, True, 1.0, layers, d, heads, K, w)
    s = torch.as_tensor(si.make_samples(L, 96, seed=2)).cuda()
    m.reset_stats()
    e = m.local_energy(s, REUSE | BF16 | INCREMENTAL)
    st = check_partition(m, 96, L * L, layers)
    assert torch.equal(e, m.local_energy(s, REUSE | BF16 | INCREMENTAL))
    ref = m.local_energy(s, REUSE).cpu().numpy().astype(np.float64)
    d_inc = rel_err(e.cpu().numpy(), ref, L * L)
    d_reuse = rel_err(m.local_energy(s, REUSE | BF16).cpu().numpy(), ref, L * L)
    print(f"8x8 d128 h4: certified {st['inc_certified_rows']} of {st['inc_patched_rows']}; BF16 vs FP32 reuse: "
          f"incremental median {np.median(d_inc):.2e}, reuse median {np.median(d_reuse):.2e}")
    assert np.median(d_inc) <= 2 * np.median(d_reuse) + 1e-4
    assert d_inc.max() <= 0.1


def test_ragged_matches_ragged_reuse():
    from paper_2212_11296_gb300 import INCREMENTAL, REUSE, VQNQS
    layers, d, heads, K, lmax = 3, 128, 4, 64, 12
    blob = si.make_weights(lmax * lmax, layers, d, K, seed=0)
    m = VQNQS(lmax, True, 1.0, layers, d, heads, K, blob)
    groups = [(L, torch.as_tensor(si.make_samples(L, B, seed=3 + L)).cuda()) for L, B in [(6, 20), (8, 12), (12, 6)]]
    e = m.local_energy_ragged(groups, REUSE | INCREMENTAL).cpu().numpy()
    assert m.stats()["device_status"] == 0
    e_ref = m.local_energy_ragged(groups, REUSE).cpu().numpy()
    err = np.abs(e - e_ref) / np.maximum(np.abs(e_ref), 1e-3 * 36)
    assert (err > 1e-5).mean() <= 0.05


def test_deterministic_and_graph_replay():
    from paper_2212_11296_gb300 import BF16, INCREMENTAL, REUSE, LocalEnergyGraph
    m, P, spins, s_dev = setup("10x10")
    for flags in (REUSE | INCREMENTAL, REUSE | BF16 | INCREMENTAL):
        a = m.local_energy(s_dev, flags)
        b = m.local_energy(s_dev, flags)
        assert torch.equal(a, b)
        g = LocalEnergyGraph(m, [(10, s_dev.shape[0])], flags)
        assert torch.equal(g(s_dev).clone(), a)


def test_flag_errors():
    from paper_2212_11296_gb300 import INCREMENTAL, REUSE, VQNQS, VQNQSError
    m, P, spins, s_dev = setup("4x4")
    with pytest.raises(VQNQSError):
        m.local_energy(s_dev, INCREMENTAL)  # needs REUSE
    w = si.make_weights(16, 2, 32, 16, seed=0)
    m8 = VQNQS(4, True, 1.0, 2, 32, 4, 16, w)  # head width 8
    with pytest.raises(VQNQSError):
        m8.local_energy(s_dev, REUSE | INCREMENTAL)
