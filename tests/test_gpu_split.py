"""Split-operand BF16 path (VQNQS_BF16_SPLIT) through the C ABI.

Each tensor-core product takes x = hi + lo in BF16 and sums three MMAs, so the
GEMMs and the attention carry FP32-grade error.  Checked here:
  * the GEMM alone (every epilogue, a ragged M tail) against float64 matmul:
    within 1e-5 of the largest output, against ~1e-3 for single BF16 operands;
  * local energies of the 16 x 16 workload against the stored FP64 oracle
    values on all 64 samples, raw (no sample exempted): relative error <= 2e-3
    (the BF16 bar), reuse and incremental;
  * an 8 x 8 model against the oracle run live, and reuse == full bitwise;
  * the incremental path's codeword at every row of every connected
    configuration against the non-incremental path's full search: equal
    except where the oracle's relative distance gap at the first differing
    layer is below 1e-4 (the split path's rounding reach).
Relative error denominator: max(|E_oracle|, 1e-3 N |J|).
"""
import numpy as np
import pytest
import torch

import synthetic_inputs as si
from golden_values import eloc_16x16
from oracle import hamiltonian, model

pytestmark = pytest.mark.gpu

BF16_BAR = 2e-3


def rel_err(got, want, N, J=1.0):
    return np.abs(np.asarray(got, np.float64) - want) / np.maximum(np.abs(want), 1e-3 * N * abs(J))


def split_bf16(x):
    hi = x.to(torch.bfloat16)
    lo = (x - hi.float()).to(torch.bfloat16)
    return hi, lo


@pytest.fixture(scope="module")
def small_ctx():
    from paper_2212_11296_gb300 import VQNQS
    return VQNQS(4, True, 1.0, 1, 64, 2, 4, si.make_weights(16, 1, 64, 4))


@pytest.mark.parametrize("epi", [0, 1, 2, 3, 4])
def test_split_gemm_is_fp32_grade(small_ctx, epi):
    m = small_ctx
    g = torch.Generator(device="cuda").manual_seed(3 + epi)
    M, N, K = 300, 192, 256  # three row tiles, the last one ragged
    A = torch.randn(M, K, device="cuda", generator=g)
    Bt = 0.05 * torch.randn(N, K, device="cuda", generator=g)
    bias = 0.1 * torch.randn(N, device="cuda", generator=g)
    R = torch.randn(M, N, device="cuda", generator=g) if epi == 2 else None
    ref = A.double() @ Bt.double().T + bias.double()
    if epi in (1, 4):
        ref = 0.5 * ref * (1.0 + torch.erf(ref / np.sqrt(2.0)))
    if epi == 2:
        ref = ref + R.double()
    A2 = torch.cat(split_bf16(A)).contiguous()
    Bt2 = torch.cat(split_bf16(Bt)).contiguous()
    C = m.gemm_bf16_split(A2, Bt2, bias, epilogue=epi, R=R)
    torch.cuda.synchronize()
    got = (C[:M].double() + C[M:].double()) if epi in (0, 1) else C.double()
    scale = ref.abs().max().item()
    err = (got - ref).abs().max().item() / scale
    # the same product from single BF16 operands, for scale
    C1 = m.gemm_bf16(A.to(torch.bfloat16), Bt.to(torch.bfloat16), bias, epilogue=epi, R=R)
    err1 = (C1.double() - ref).abs().max().item() / scale
    print(f"epilogue {epi}: split {err:.2e}, single BF16 {err1:.2e}")
    assert err <= 1e-5
    assert err1 > 20 * err


@pytest.fixture(scope="module")
def ctx16():
    from paper_2212_11296_gb300 import VQNQS
    L, layers, d, heads, K = 16, 8, 256, 8, 256
    N = L * L
    w = si.make_weights(N, layers, d, K, seed=0)
    spins = si.make_samples(L, 64, seed=1)
    m = VQNQS(L, True, 1.0, layers, d, heads, K, w)
    return m, spins, torch.as_tensor(spins).cuda()


@pytest.mark.parametrize("incremental", [False, True])
def test_16x16_split_within_bf16_bar_of_oracle_raw(ctx16, incremental):
    from paper_2212_11296_gb300 import BF16, BF16_SPLIT, INCREMENTAL, REUSE
    m, spins, s_dev = ctx16
    want, _, gap = eloc_16x16()
    flags = REUSE | BF16 | BF16_SPLIT | (INCREMENTAL if incremental else 0)
    m.reset_stats()
    got = m.local_energy(s_dev, flags).cpu().numpy()
    assert m.stats()["device_status"] == 0
    err = rel_err(got, want, 256)
    plain = rel_err(m.local_energy(s_dev, REUSE | BF16 | (INCREMENTAL if incremental else 0)).cpu().numpy(),
                    want, 256)
    print(f"split: max {err.max():.2e} median {np.median(err):.2e}; "
          f"single BF16: max {plain.max():.2e} median {np.median(plain):.2e}")
    assert err.max() <= BF16_BAR, np.argsort(-err)[:5]
    assert np.median(err) <= 1e-5


def test_8x8_split_matches_oracle_and_reuse_equals_full():
    from paper_2212_11296_gb300 import BF16, BF16_SPLIT, INCREMENTAL, REUSE, VQNQS
    L, layers, d, heads, K, B = 8, 2, 128, 4, 64, 24
    N = L * L
    w = si.make_weights(N, layers, d, K, seed=0)
    spins = si.make_samples(L, B, seed=1)
    m = VQNQS(L, True, 1.0, layers, d, heads, K, w)
    P = model.parse_blob(w, N, layers, d, heads, K)
    s_dev = torch.as_tensor(spins).cuda()
    want = hamiltonian.local_energy(P, spins, L, True, 1.0)
    full = m.local_energy(s_dev, BF16 | BF16_SPLIT)
    reuse = m.local_energy(s_dev, REUSE | BF16 | BF16_SPLIT)
    inc = m.local_energy(s_dev, REUSE | BF16 | BF16_SPLIT | INCREMENTAL)
    assert torch.equal(full, reuse)
    for got in (reuse, inc):
        err = rel_err(got.cpu().numpy(), want, N)
        print(f"max {err.max():.2e} median {np.median(err):.2e}")
        assert err.max() <= BF16_BAR and np.median(err) <= 1e-5


def test_split_flag_validation():
    from paper_2212_11296_gb300 import BF16_SPLIT, REUSE, VQNQS, VQNQSError
    m = VQNQS(4, True, 1.0, 1, 64, 2, 4, si.make_weights(16, 1, 64, 4))
    s = torch.zeros(2, 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(VQNQSError, match="ERR_ARG"):
        m.local_energy(s, REUSE | BF16_SPLIT)  # needs BF16


def test_incremental_split_codes_equal_full_search(ctx16):
    """Every connected configuration's codeword at every layer and position from
    the incremental path (certified or searched) against the non-incremental
    path (every row searched), 4 samples (about 1000 configurations, 2 M
    assignments).  Where they differ, the first differing layer's rows must be
    oracle near ties (relative gap < 1e-4): there the two computations' FP32-grade
    rounding may legitimately pick different codewords."""
    from paper_2212_11296_gb300 import BF16, BF16_SPLIT, INCREMENTAL, REUSE
    m, spins, s_dev = ctx16
    sub = s_dev[:4].contiguous()
    e_inc, c_inc = m.local_energy_codes(sub, REUSE | BF16 | BF16_SPLIT | INCREMENTAL)
    e_ful, c_ful = m.local_energy_codes(sub, REUSE | BF16 | BF16_SPLIT)
    c_inc, c_ful = c_inc.cpu().numpy(), c_ful.cpu().numpy()
    assert np.array_equal(c_inc < 0, c_ful < 0)
    valid = c_ful[:, :, 0, 0] >= 0
    diff = (c_inc != c_ful) & valid[:, :, None, None]
    n_assign = int(valid.sum()) * m.layers * m.N
    print(f"{int(diff.sum())} of {n_assign} assignments differ")
    assert diff.sum() <= 1e-4 * n_assign
    if diff.any():
        P = model.parse_blob(si.make_weights(256, 8, 256, 256, seed=0), 256, 8, 256, 8, 256)
        bl = hamiltonian.bonds(16, True)
        for b, k in zip(*np.nonzero(diff.any(axis=(2, 3)))):
            _, cfgs, _ = hamiltonian.connected(spins[b], bl, 1.0)
            cfg = spins[b][None] if k == 0 else cfgs[k - 1][None]
            gaps = []
            model.forward(P, cfg, gaps=gaps)
            l = int(np.nonzero(diff[b, k].any(axis=1))[0][0])
            rows = np.nonzero(diff[b, k, l])[0]
            g = gaps[l][0].numpy()[rows]
            print(f"sample {b} configuration {k} layer {l} rows {rows}: oracle gaps {g}")
            assert np.all(g < 1e-4)


def test_incremental_work_split_tuner_keeps_results(ctx16):
    """vqnqs_autotune_incremental only reassigns work to CTAs: the local energies after it
    (with the chosen split) equal those before it bitwise, and the choices are the offered ones."""
    from paper_2212_11296_gb300 import BF16, BF16_SPLIT, INCREMENTAL, REUSE
    m, spins, s_dev = ctx16
    flags = REUSE | BF16 | BF16_SPLIT | INCREMENTAL
    sub = s_dev[:8].contiguous()
    before = m.local_energy(sub, flags)
    t = m.autotune_incremental(sub, flags)
    print(t)
    assert t["patch_items"] in (2, 4, 8) and t["rows_slices"] in (1, 2, 4, 8, 16)
    assert all(v > 0 for v in t["patch_ms"].values()) and all(v > 0 for v in t["rows_ms"].values())
    assert torch.equal(m.local_energy(sub, flags), before)
    assert m.stats()["device_status"] == 0
