"""Seeded synthetic inputs for the VQ-NQS local-energy path.

This module holds only random-number generation and the flat weight-blob
layout used to place the random values; it contains none of the method's
arithmetic (no model, no Hamiltonian).  Both the oracle and the CUDA path are
fed from here, which is the only code they share.

Generator (counter based, documented so any language can reproduce it):

* ``splitmix64(seed, i)``: z = seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64),
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9, z = (z ^ (z >> 27)) *
  0x94D049BB133111EB, return z ^ (z >> 31).
* uniform u in [0, 1): (z >> 11) * 2^-53.
* normal pairs by Box-Muller: for k = 0, 1, ...: u1 = uniform(2k),
  u2 = uniform(2k + 1); r = sqrt(-2 ln(1 - u1)); value 2k = r cos(2 pi u2),
  value 2k + 1 = r sin(2 pi u2).

Weights: every blob entry i is std * normal(i) with std = 0.02 (seed 0 by
default); then every bias and LayerNorm shift is set to 0 and every LayerNorm
gain to 1.

Samples: uniform random S_z = 0 configurations.  Sample b draws N uniforms
from the stream with seed ``seed * 2^32 + b`` and marks the N/2 sites holding
the smallest keys as up (1); the rest are down (0).  Every balanced
configuration is equally likely.  Spins are raster ordered, p = y * L + x.

Weight blob layout (float32, in this order; d = d_model, n_max = max sites):
  tok_emb[3, d]            rows: token 0 = down, 1 = up, 2 = begin-of-sequence
  pos_emb[n_max, d]
  per layer l = 0 .. layers-1:
    ln1_g[d], ln1_b[d]
    w_qkv[d, 3d], b_qkv[3d]          a @ w_qkv; columns [q | k | v]
    codebook[K, d]
    w_o[d, d], b_o[d]
    ln2_g[d], ln2_b[d]
    w_1[d, 4d], b_1[4d]
    w_2[4d, d], b_2[d]
  lnf_g[d], lnf_b[d], w_head[d, 2], b_head[2]
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based splitmix64: one 64-bit output per counter value."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, n: int, start: int = 0) -> np.ndarray:
    z = splitmix64(seed, np.arange(start, start + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller over the uniform stream."""
    m = (n + 1) // 2
    u = uniforms(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    t = 2.0 * np.pi * u2
    out = np.empty(2 * m, dtype=np.float64)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:n]


def blob_segments(n_max: int, layers: int, d: int, K: int, half_block: bool = False, token_group: int = 1):
    """(name, shape, kind) for every tensor of the blob, in order.

    kind is 'w' (random), 'zero' (bias / LayerNorm shift) or 'one' (gain).  With
    half_block the final attention-only half-block (LN, W_qkv, W_o and their
    biases) follows the quantized blocks.  With token_group G each token is a
    group of G spins: 2^G + 1 token embeddings (the last one begin-of-sequence),
    n_max / G positions and a 2^G-way head."""
    G = token_group
    seg = [("tok_emb", ((1 << G) + 1, d), "w"), ("pos_emb", (n_max // G, d), "w")]
    for l in range(layers):
        p = f"l{l}."
        seg += [
            (p + "ln1_g", (d,), "one"), (p + "ln1_b", (d,), "zero"),
            (p + "w_qkv", (d, 3 * d), "w"), (p + "b_qkv", (3 * d,), "zero"),
            (p + "codebook", (K, d), "w"),
            (p + "w_o", (d, d), "w"), (p + "b_o", (d,), "zero"),
            (p + "ln2_g", (d,), "one"), (p + "ln2_b", (d,), "zero"),
            (p + "w_1", (d, 4 * d), "w"), (p + "b_1", (4 * d,), "zero"),
            (p + "w_2", (4 * d, d), "w"), (p + "b_2", (d,), "zero"),
        ]
    if half_block:
        seg += [("h.ln_g", (d,), "one"), ("h.ln_b", (d,), "zero"),
                ("h.w_qkv", (d, 3 * d), "w"), ("h.b_qkv", (3 * d,), "zero"),
                ("h.w_o", (d, d), "w"), ("h.b_o", (d,), "zero")]
    seg += [("lnf_g", (d,), "one"), ("lnf_b", (d,), "zero"),
            ("w_head", (d, 1 << G), "w"), ("b_head", (1 << G,), "zero")]
    return seg


def num_params(n_max: int, layers: int, d: int, K: int, half_block: bool = False, token_group: int = 1) -> int:
    return int(sum(int(np.prod(s)) for _, s, _ in blob_segments(n_max, layers, d, K, half_block, token_group)))


def make_weights(n_max: int, layers: int, d: int, K: int, seed: int = 0,
                 std: float = 0.02, half_block: bool = False, token_group: int = 1) -> np.ndarray:
    """Seeded float32 weight blob in the layout documented above."""
    n = num_params(n_max, layers, d, K, half_block, token_group)
    blob = (std * normals(seed, n)).astype(np.float32)
    off = 0
    for _, shape, kind in blob_segments(n_max, layers, d, K, half_block, token_group):
        sz = int(np.prod(shape))
        if kind == "zero":
            blob[off:off + sz] = 0.0
        elif kind == "one":
            blob[off:off + sz] = 1.0
        off += sz
    return blob


def make_samples(L: int, B: int, seed: int = 1) -> np.ndarray:
    """B uniform random S_z = 0 spin configurations of an L x L lattice, uint8 [B, N]."""
    N = L * L
    if N % 2:
        raise ValueError("S_z = 0 needs an even number of sites")
    out = np.zeros((B, N), dtype=np.uint8)
    for b in range(B):
        keys = uniforms((seed << 32) + b, N)
        up = np.argsort(keys, kind="stable")[: N // 2]
        out[b, up] = 1
    return out


def make_chain_samples(N: int, B: int, seed: int = 1) -> np.ndarray:
    """B configurations of an N-site chain with independent uniform spins, uint8 [B, N]
    (spin p of sample b is up when uniform number p of stream seed * 2^32 + b is below 1/2)."""
    out = np.zeros((B, N), dtype=np.uint8)
    for b in range(B):
        out[b] = (uniforms((seed << 32) + b, N) < 0.5).astype(np.uint8)
    return out
