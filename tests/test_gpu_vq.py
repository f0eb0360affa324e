"""Nearest-codeword kernels through the C ABI (vqnqs_vq_assign): the FP32 FFMA
kernel and the tensor-core kernel (split-TF32 products) against an FP64
brute-force argmin on the host.  Both must agree with FP64 on every row whose
relative gap (l2 - l1) / l1 between the two smallest squared distances is at
least 1e-6, and exact ties must go to the lowest index."""
import numpy as np
import pytest
import torch

import synthetic_inputs as si
from oracle import model

pytestmark = pytest.mark.gpu


def make(d, K, layers=1, seed=0):
    from paper_2212_11296_gb300 import VQNQS
    w = si.make_weights(16, layers, d, K, seed=seed)
    return VQNQS(4, True, 1.0, layers, d, max(1, d // 32), K, w), model.parse_blob(w, 16, layers, d, max(1, d // 32), K)


def fp64_assign(O, W):
    d2 = (O ** 2).sum(1, keepdims=True) - 2 * O @ W.T + (W ** 2).sum(1)
    order = np.argsort(d2, axis=1, kind="stable")
    l1 = d2[np.arange(len(O)), order[:, 0]]
    l2 = d2[np.arange(len(O)), order[:, 1]]
    return order[:, 0], (l2 - l1) / np.maximum(l1, 1e-30)


@pytest.mark.parametrize("d,K", [(64, 16), (128, 64), (256, 256), (384, 512), (192, 128)])
@pytest.mark.parametrize("tc", [False, True])
def test_assign_matches_fp64(d, K, tc):
    m, P = make(d, K)
    W = P.t["0.codebook"].numpy()
    rng = np.random.default_rng(d + K)
    R = 5000
    # attention outputs: codeword-scale vectors plus an offset common to all rows
    O = (rng.standard_normal((R, d)) * 0.3 + rng.standard_normal(d) * 0.5).astype(np.float32)
    code = m.vq_assign(0, torch.as_tensor(O).cuda(), tensor_cores=tc).cpu().numpy()
    want, gap = fp64_assign(O.astype(np.float64), W.astype(np.float64))
    clear = gap >= 1e-6
    assert clear.mean() > 0.95
    assert np.array_equal(code[clear], want[clear]), np.nonzero(code[clear] != want[clear])[0][:10]


@pytest.mark.parametrize("tc", [False, True])
def test_assign_exact_ties_lowest_index(tc):
    from paper_2212_11296_gb300 import VQNQS
    d, K = 64, 16
    w = si.make_weights(16, 1, d, K, seed=3)
    P = model.parse_blob(w, 16, 1, d, 2, K)
    cb = P.t["0.codebook"]
    cb[8:] = cb[:8]  # codeword j + 8 repeats codeword j
    blob = np.concatenate([P.t[k].numpy().ravel() for k in P.t]).astype(np.float32)
    m = VQNQS(4, True, 1.0, 1, d, 2, K, blob)
    O = np.random.default_rng(0).standard_normal((777, d)).astype(np.float32) * 0.05
    code = m.vq_assign(0, torch.as_tensor(O).cuda(), tensor_cores=tc).cpu().numpy()
    assert np.all(code < 8)
    want, _ = fp64_assign(O.astype(np.float64), cb.numpy())
    assert np.array_equal(code, want)


def test_tensor_core_and_ffma_agree_off_ties():
    m, P = make(256, 256)
    rng = np.random.default_rng(5)
    O = torch.as_tensor((rng.standard_normal((100000, 256)) * 0.2).astype(np.float32)).cuda()
    a = m.vq_assign(0, O, tensor_cores=False)
    b = m.vq_assign(0, O, tensor_cores=True)
    assert (a != b).float().mean().item() < 1e-4
    assert m.stats()["device_status"] == 0
