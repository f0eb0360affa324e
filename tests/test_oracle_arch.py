"""Pins of the oracle's architecture variants (Sec. 3.1 and Table 1): the
multi-head quantizer (Eq. vq with H heads), the final half-block and tokens
of G spins.

* Brute force: the quantized vector is the joint nearest point over all K^H
  concatenations of one codeword per segment (the squared distance splits into
  one term per segment), found here by enumerating every tuple.
* Scalar segments (H = d): each coordinate goes to its nearest codebook value
  (closed form).
* With K = 1 the codebook block [H, 1, d/H] is the same memory as a single
  codeword [1, d]: the model read with H heads equals the one-head model.
* The multi-head model is a normalised autoregressive distribution.
"""
import itertools

import numpy as np
import pytest
import torch

import synthetic_inputs as si
from oracle import model


@pytest.mark.parametrize("H,K,dq", [(2, 4, 4), (3, 3, 2), (4, 2, 3)])
def test_quantize_is_joint_nearest_by_brute_force(H, K, dq):
    g = torch.Generator().manual_seed(H * 100 + K * 10 + dq)
    cb = torch.randn(H, K, dq, generator=g, dtype=torch.float64)
    o = torch.randn(7, H * dq, generator=g, dtype=torch.float64)
    V, codes = model.quantize(o, cb)
    for r in range(o.shape[0]):
        best, arg = None, None
        for tup in itertools.product(range(K), repeat=H):
            v = torch.cat([cb[h, tup[h]] for h in range(H)])
            dist = float(((o[r] - v) ** 2).sum())
            if best is None or dist < best:
                best, arg = dist, tup
        assert tuple(int(c) for c in codes[r]) == arg
        assert torch.equal(V[r], torch.cat([cb[h, arg[h]] for h in range(H)]))


def test_scalar_segments_closed_form():
    d, K = 6, 5
    rng = np.random.default_rng(3)
    cb = rng.standard_normal((d, K, 1))
    o = rng.standard_normal((9, d))
    V, codes = model.quantize(torch.as_tensor(o), torch.as_tensor(cb))
    want_idx = np.argmin(np.abs(o[:, :, None] - cb[None, :, :, 0]), axis=-1)
    assert np.array_equal(codes.numpy(), want_idx)
    assert np.allclose(V.numpy(), np.take_along_axis(cb[None, :, :, 0].repeat(9, 0), want_idx[..., None], -1)[..., 0],
                       rtol=0, atol=0)


def test_single_head_path_unchanged():
    g = torch.Generator().manual_seed(5)
    cb = torch.randn(6, 8, generator=g, dtype=torch.float64)
    o = torch.randn(11, 8, generator=g, dtype=torch.float64)
    V, codes = model.quantize(o, cb)
    c = model.nearest_code(o, cb)
    assert torch.equal(codes[:, 0], c) and torch.equal(V, cb[c])


@pytest.mark.parametrize("H", [2, 4])
def test_one_code_per_head_equals_single_head_model(H):
    L, layers, d, heads = 4, 2, 16, 2
    N = L * L
    w = si.make_weights(N, layers, d, 1, seed=4, std=0.3)
    P1 = model.parse_blob(w, N, layers, d, heads, 1)
    PH = model.parse_blob(w, N, layers, d, heads, 1, vq_heads=H)
    spins = si.make_samples(L, 12, seed=2)
    assert np.array_equal(model.log_psi(P1, spins), model.log_psi(PH, spins))


def test_multi_head_model_is_normalised():
    N, layers, d, heads, K, H = 4, 2, 16, 2, 4, 4
    w = si.make_weights(N, layers, d, K, seed=6, std=0.4)
    P = model.parse_blob(w, N, layers, d, heads, K, vq_heads=H)
    states = np.array(list(itertools.product([0, 1], repeat=N)))
    lp = model.log_psi(P, states)
    assert abs(np.exp(2.0 * lp).sum() - 1.0) < 1e-12
    # several heads do change the model when K > 1
    P1 = model.parse_blob(w, N, layers, d, heads, K)
    assert not np.allclose(lp, model.log_psi(P1, states))


def _zero_half_block_blob(N, layers, d, K, seed, std=0.3):
    """The blob of a half-block model whose W_o and b_o are zero, and the blob of the
    same network without the half-block."""
    w_h = si.make_weights(N, layers, d, K, seed=seed, std=std, half_block=True)
    off = 0
    for name, shape, _ in si.blob_segments(N, layers, d, K, half_block=True):
        sz = int(np.prod(shape))
        if name in ("h.w_o", "h.b_o"):
            w_h[off:off + sz] = 0.0
        off += sz
    keep = []
    off = 0
    for name, shape, _ in si.blob_segments(N, layers, d, K, half_block=True):
        sz = int(np.prod(shape))
        if not name.startswith("h."):
            keep.append(w_h[off:off + sz])
        off += sz
    return w_h, np.concatenate(keep)


def test_half_block_with_zero_projection_is_the_plain_model():
    L, layers, d, heads, K = 4, 2, 16, 2, 4
    N = L * L
    w_h, w = _zero_half_block_blob(N, layers, d, K, seed=8)
    Ph = model.parse_blob(w_h, N, layers, d, heads, K, half_block=True)
    P = model.parse_blob(w, N, layers, d, heads, K)
    spins = si.make_samples(L, 10, seed=3)
    assert np.array_equal(model.log_psi(Ph, spins), model.log_psi(P, spins))


def test_half_block_model_is_normalised_and_differs():
    N, layers, d, heads, K = 4, 2, 16, 2, 4
    w = si.make_weights(N, layers, d, K, seed=9, std=0.4, half_block=True)
    P = model.parse_blob(w, N, layers, d, heads, K, vq_heads=2, half_block=True)
    states = np.array(list(itertools.product([0, 1], repeat=N)))
    lp = model.log_psi(P, states)
    assert abs(np.exp(2.0 * lp).sum() - 1.0) < 1e-12
    w_h, w0 = _zero_half_block_blob(N, layers, d, K, seed=9, std=0.4)  # the same network, W_o = 0
    assert not np.allclose(lp, model.log_psi(model.parse_blob(w0, N, layers, d, heads, K, vq_heads=2), states))


def _passthrough_blob(N, layers, d, K, G, seed):
    """A G-token blob whose blocks leave x unchanged (W_o, b_o, W_2, b_2 zero)."""
    w = si.make_weights(N, layers, d, K, seed=seed, std=0.5, token_group=G)
    off = 0
    for name, shape, _ in si.blob_segments(N, layers, d, K, token_group=G):
        sz = int(np.prod(shape))
        if name.endswith((".w_o", ".b_o", ".w_2", ".b_2")):
            w[off:off + sz] = 0.0
        off += sz
    return w


@pytest.mark.parametrize("G", [2, 4])
def test_token_groups_closed_form_without_blocks(G):
    """With blocks that pass x through, P(group t | earlier) is the head applied to
    tok_emb[value of group t-1 (BOS 2^G at t = 0)] + pos_emb[t], computed here in numpy."""
    N, layers, d, heads, K = 8, 2, 16, 2, 4
    w = _passthrough_blob(N, layers, d, K, G, seed=11)
    P = model.parse_blob(w, N, layers, d, heads, K, token_group=G)
    seg = {name: shape for name, shape, _ in si.blob_segments(N, layers, d, K, token_group=G)}
    off, arr = 0, {}
    for name, shape, _ in si.blob_segments(N, layers, d, K, token_group=G):
        sz = int(np.prod(shape))
        arr[name] = w[off:off + sz].astype(np.float64).reshape(shape)
        off += sz
    rng = np.random.default_rng(G)
    spins = rng.integers(0, 2, size=(6, N)).astype(np.uint8)
    T = N // G
    want = np.zeros(len(spins))
    for b, s in enumerate(spins):
        vals = [sum(int(s[t * G + k]) << k for k in range(G)) for t in range(T)]
        for t in range(T):
            tok = (1 << G) if t == 0 else vals[t - 1]
            x = arr["tok_emb"][tok] + arr["pos_emb"][t]
            a = (x - x.mean()) / np.sqrt(x.var() + 1e-5) * arr["lnf_g"] + arr["lnf_b"]
            z = a @ arr["w_head"] + arr["b_head"]
            lse = z.max() + np.log(np.exp(z - z.max()).sum())
            want[b] += 0.5 * (z[vals[t]] - lse)
    assert seg["w_head"] == (d, 1 << G)
    assert np.allclose(model.log_psi(P, spins), want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("G", [2, 4])
def test_token_group_model_is_normalised(G):
    N, layers, d, heads, K = 4, 2, 16, 2, 4
    w = si.make_weights(N, layers, d, K, seed=12, std=0.4, token_group=G)
    P = model.parse_blob(w, N, layers, d, heads, K, vq_heads=2, token_group=G)
    states = np.array(list(itertools.product([0, 1], repeat=N)))
    assert abs(np.exp(2.0 * model.log_psi(P, states)).sum() - 1.0) < 1e-12


def test_st_gradient_of_the_variants_matches_finite_differences():
    """Eq. st per quantizer head, with the half-block and tokens of two spins:
    central differences (h = 1e-6) of the straight-through surrogate, its
    stop-gradient terms frozen at theta_0, equal the autograd O_k."""
    import dataclasses
    from oracle import gradient
    L, layers, d, heads, K, H, G = 4, 2, 16, 2, 4, 2, 2
    N = L * L
    w = si.make_weights(N, layers, d, K, seed=13, std=0.3, half_block=True, token_group=G)
    P = model.parse_blob(w, N, layers, d, heads, K, vq_heads=H, half_block=True, token_group=G)
    s = si.make_samples(L, 1, seed=9)
    O = gradient.per_sample_O(P, s)[0]
    frozen = gradient.record_frozen(P, s)
    names = list(P.t)
    sizes = [P.t[n].numel() for n in names]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(5)
    picks = list(rng.choice(len(O), 120, replace=False))
    for n in ("0.codebook", "1.codebook", "h.w_o", "h.w_qkv", "w_head", "tok_emb"):
        k = names.index(n)
        picks += list(range(offs[k], min(offs[k] + 8, offs[k + 1])))
    h = 1e-6
    for g in picks:
        k = int(np.searchsorted(offs, g, side="right") - 1)
        name, j = names[k], int(g - offs[k])
        vals = []
        for sgn in (+1, -1):
            Q = dataclasses.replace(P, t={a: b.clone() for a, b in P.t.items()})
            Q.t[name].view(-1)[j] += sgn * h
            with torch.no_grad():
                vals.append(float(gradient.log_psi_with(Q, s, gradient.frozen_quantizer(Q, frozen))[0]))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - O[g]) <= 1e-7 * max(1.0, abs(O[g])), (name, j, fd, O[g])
    # the codebooks do receive a gradient through softmax(D_h) of each head
    k = names.index("0.codebook")
    assert np.abs(O[offs[k]:offs[k + 1]]).max() > 0
