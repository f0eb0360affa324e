"""Oracle: the VQ-NQS autoregressive wave function, float64 on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What it computes (Sec. 2 polar form and chain rule; Sec. 3.1 architecture;
Sec. 4 phase set to zero by the Marshall sign rule):

  psi(s) = sqrt(P(s)),  P(s) = prod_p P(s_p | s_<p),
  log psi(s) = 1/2 * sum_p log P(s_p | s_<p).

P is a decoder (causal) transformer with one token per spin.  The input at
position p is the previous spin s_{p-1} (a begin-of-sequence token at p = 0),
so the output at p is the conditional of s_p.  Each block is pre-LayerNorm:

  a = LN1(x);  q, k, v = a W_qkv + b_qkv
  o = causal multi-head softmax(q k^T / sqrt(d/heads)) v       (location mixer)
  c = argmin_j ||o - W_j||^2, lowest j on ties                  (Eq. vq)
  y = x + W_o W_c + b_o            (the quantizer sits after the attention,
                                    before the output projection and residual)
  x <- y + W_2 GELU(W_1 LN2(y) + b_1) + b_2                     (per location)

and the head is log_softmax(LN_f(x) W_head + b_head) over the two spin values.
LayerNorm uses eps = 1e-5 and the biased variance; GELU is the erf form.

Tokens as particle groups (Sec. 3.1): with token_group G each token is a group
of G consecutive spins with value sum_k s[tG + k] 2^k, the input at position t
is the value of group t - 1 (begin-of-sequence 2^G at t = 0), the head is a
2^G-way log-softmax and log psi = 1/2 sum_t log P(group t | earlier groups).

Optional final half-block (Table 1's networks): after the blocks,
x <- x + W_o attention(LN(x)) + b_o with its own weights and no quantizer.

Multi-head VQ (Eq. vq with H heads): o is split into H segments of d/H
values, segment h is quantized with its own codebook W_h of K vectors (the
codebook block of the blob is W in R^{H x K x d/H}), and the quantized vector
is the concatenation of the chosen W_h rows; H = 1 is the single-head case.

Readings of the paper used here (it leaves block internals to prior work):
pre-LN, erf-GELU, biases everywhere, and the argmax in Eq. vq read as the
argmax of D = -||x_h - W_h,j||, i.e. the nearest codeword of each segment.  The squared distance is expanded as ||o||^2 - 2 o.W_j + ||W_j||^2 in
float64; its argmin equals the direct one unless two distances agree to ~1e-15
relative.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

LN_EPS = 1e-5
BOS = 2


@dataclass
class Params:
    d: int
    heads: int
    K: int
    layers: int
    n_max: int
    t: dict  # name -> float64 tensor
    vq_heads: int = 1
    half_block: bool = False
    token_group: int = 1  # G spins per token (Sec. 3.1 tokens as particle groups)


def parse_blob(blob, n_max: int, layers: int, d: int, heads: int, K: int, vq_heads: int = 1,
               half_block: bool = False, token_group: int = 1) -> Params:
    """Split a flat float32 weight blob into named float64 tensors.

    The order is the documented blob order: token and position embeddings,
    then per layer LN1, W_qkv, codebook, W_o, LN2, W_1, W_2 (each matrix
    followed by its bias), then LN_f and the head.  The codebook block holds
    K * d values: [K, d] for one quantizer head, [vq_heads, K, d / vq_heads]
    for several.  With half_block, LN, W_qkv and W_o of the final
    attention-only half-block follow the blocks."""
    if d % vq_heads:
        raise ValueError("d must be a multiple of vq_heads")
    blob = torch.as_tensor(np.asarray(blob, dtype=np.float32)).double()
    pos = 0
    t = {}

    def take(name, *shape):
        nonlocal pos
        n = int(np.prod(shape))
        t[name] = blob[pos:pos + n].reshape(shape).clone()
        pos += n

    G = token_group
    if n_max % G:
        raise ValueError("n_max must be a multiple of token_group")
    take("tok_emb", (1 << G) + 1, d)
    take("pos_emb", n_max // G, d)
    for l in range(layers):
        take(f"{l}.ln1_g", d); take(f"{l}.ln1_b", d)
        take(f"{l}.w_qkv", d, 3 * d); take(f"{l}.b_qkv", 3 * d)
        if vq_heads == 1:
            take(f"{l}.codebook", K, d)
        else:
            take(f"{l}.codebook", vq_heads, K, d // vq_heads)
        take(f"{l}.w_o", d, d); take(f"{l}.b_o", d)
        take(f"{l}.ln2_g", d); take(f"{l}.ln2_b", d)
        take(f"{l}.w_1", d, 4 * d); take(f"{l}.b_1", 4 * d)
        take(f"{l}.w_2", 4 * d, d); take(f"{l}.b_2", d)
    if half_block:
        take("h.ln_g", d); take("h.ln_b", d)
        take("h.w_qkv", d, 3 * d); take("h.b_qkv", 3 * d)
        take("h.w_o", d, d); take("h.b_o", d)
    take("lnf_g", d); take("lnf_b", d)
    take("w_head", d, 1 << G); take("b_head", 1 << G)
    if pos != blob.numel():
        raise ValueError(f"blob has {blob.numel()} values, layout needs {pos}")
    return Params(d=d, heads=heads, K=K, layers=layers, n_max=n_max, t=t, vq_heads=vq_heads,
                  half_block=half_block, token_group=G)


def layer_norm(x, g, b):
    mu = x.mean(dim=-1, keepdim=True)
    var = ((x - mu) ** 2).mean(dim=-1, keepdim=True)
    return (x - mu) / torch.sqrt(var + LN_EPS) * g + b


def gelu(x):
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def causal_attention(a, w_qkv, b_qkv, heads):
    """Causal multi-head self-attention output before the output projection.

    a: [C, N, d] -> o: [C, N, d] (heads concatenated)."""
    C, N, d = a.shape
    dh = d // heads
    qkv = a @ w_qkv + b_qkv
    q, k, v = qkv[..., :d], qkv[..., d:2 * d], qkv[..., 2 * d:]
    q = q.reshape(C, N, heads, dh).transpose(1, 2)
    k = k.reshape(C, N, heads, dh).transpose(1, 2)
    v = v.reshape(C, N, heads, dh).transpose(1, 2)
    scores = (q @ k.transpose(-1, -2)) / math.sqrt(dh)
    future = torch.ones(N, N, dtype=torch.bool).triu(1)
    scores = scores.masked_fill(future, float("-inf"))
    p = torch.softmax(scores, dim=-1)
    o = p @ v
    return o.transpose(1, 2).reshape(C, N, d)


def sq_distances(o, codebook):
    """||o - W_j||^2 for every row of o and every codeword j."""
    return (o * o).sum(-1, keepdim=True) - 2.0 * (o @ codebook.T) + (codebook * codebook).sum(-1)


def nearest_code(o, codebook):
    """Eq. vq: index of the nearest codeword, lowest index on exact ties."""
    return torch.argmin(sq_distances(o, codebook), dim=-1)


def quantize(o, codebook):
    """Eq. vq with H heads.  codebook [K, d] (H = 1) or [H, K, d / H].

    Returns (V, codes): V the concatenation over h of W_h[c_h], codes [..., H]
    with c_h the nearest codeword of segment h (lowest index on exact ties)."""
    if codebook.dim() == 2:
        c = nearest_code(o, codebook)
        return codebook[c], c[..., None]
    H, K, dq = codebook.shape
    parts, codes = [], []
    for h in range(H):
        seg = o[..., h * dq:(h + 1) * dq]
        c = nearest_code(seg, codebook[h])
        parts.append(codebook[h][c])
        codes.append(c)
    return torch.cat(parts, dim=-1), torch.stack(codes, dim=-1)


def segment_gap(o, codebook):
    """Smallest relative_gap over the quantizer's segments."""
    if codebook.dim() == 2:
        return relative_gap(o, codebook)
    H, K, dq = codebook.shape
    return torch.stack([relative_gap(o[..., h * dq:(h + 1) * dq], codebook[h]) for h in range(H)]).min(0).values


def group_values(spins: torch.Tensor, G: int = 1) -> torch.Tensor:
    """Value of each group of G consecutive spins, sum_k s[t G + k] 2^k: [C, N / G]."""
    C, N = spins.shape
    g = spins.long().reshape(C, N // G, G)
    return (g * (1 << torch.arange(G))).sum(-1)


def tokens(spins: torch.Tensor, G: int = 1) -> torch.Tensor:
    """Shift right: the token at position t is the value of group t - 1, the
    begin-of-sequence token 2^G at t = 0 (for G = 1: s_{p-1}, BOS = 2)."""
    v = group_values(spins, G)
    tok = torch.empty_like(v)
    tok[:, 0] = 1 << G
    tok[:, 1:] = v[:, :-1]
    return tok


def relative_gap(o, codebook):
    """(l2 - l1) / l1 for the two smallest squared distances l1 <= l2 of each row
    (diagnostic: how close a row is to a codeword tie)."""
    if codebook.shape[0] < 2:
        return torch.full(o.shape[:-1], float("inf"), dtype=o.dtype)
    d2 = torch.topk(sq_distances(o, codebook), 2, dim=-1, largest=False).values
    return (d2[..., 1] - d2[..., 0]) / torch.clamp(d2[..., 0], min=1e-30)


def forward(P: Params, spins, quantizer=None, record=None, gaps=None):
    """Conditional log-probabilities log P(. | earlier groups), shape [C, N / G, 2^G].

    ``quantizer(l, o) -> (V, codes)`` replaces the plain nearest-codeword
    lookup (used by the gradient module for the straight-through form);
    ``record`` (a list) receives the codes of every layer and ``gaps`` (a
    list) the per-row relative gap of every layer."""
    spins = torch.as_tensor(np.asarray(spins)).long()
    C, N = spins.shape
    t = P.t
    T = N // P.token_group
    x = t["tok_emb"][tokens(spins, P.token_group)] + t["pos_emb"][:T]
    for l in range(P.layers):
        a = layer_norm(x, t[f"{l}.ln1_g"], t[f"{l}.ln1_b"])
        o = causal_attention(a, t[f"{l}.w_qkv"], t[f"{l}.b_qkv"], P.heads)
        if quantizer is None:
            vq, c = quantize(o, t[f"{l}.codebook"])
            if P.vq_heads == 1:
                c = c[..., 0]
        else:
            vq, c = quantizer(l, o)
        if record is not None:
            record.append(c)
        if gaps is not None:
            gaps.append(segment_gap(o, t[f"{l}.codebook"]))
        y = x + vq @ t[f"{l}.w_o"] + t[f"{l}.b_o"]
        h = gelu(layer_norm(y, t[f"{l}.ln2_g"], t[f"{l}.ln2_b"]) @ t[f"{l}.w_1"] + t[f"{l}.b_1"])
        x = y + h @ t[f"{l}.w_2"] + t[f"{l}.b_2"]
    if P.half_block:  # Table 1's final half-block: attention and W_o, no quantizer, no MLP
        a = layer_norm(x, t["h.ln_g"], t["h.ln_b"])
        o = causal_attention(a, t["h.w_qkv"], t["h.b_qkv"], P.heads)
        x = x + o @ t["h.w_o"] + t["h.b_o"]
    logits = layer_norm(x, t["lnf_g"], t["lnf_b"]) @ t["w_head"] + t["b_head"]
    return torch.log_softmax(logits, dim=-1)


def log_psi(P: Params, spins, batch: int = 64, record=None, min_gap=None) -> np.ndarray:
    """log psi(s) = 1/2 sum_p log P(s_p | s_<p) for each row of ``spins`` (float64).

    ``min_gap`` (a float64 array of len(spins)) receives, per configuration, the
    smallest relative codeword gap over all its rows and layers."""
    spins = np.asarray(spins)
    out = np.empty(spins.shape[0], dtype=np.float64)
    with torch.no_grad():
        for i in range(0, spins.shape[0], batch):
            s = torch.as_tensor(spins[i:i + batch]).long()
            rec = [] if record is not None else None
            gp = [] if min_gap is not None else None
            lp = forward(P, s, record=rec, gaps=gp)
            v = group_values(s, P.token_group)
            out[i:i + batch] = 0.5 * lp.gather(-1, v[..., None])[..., 0].sum(-1).numpy()
            if record is not None:
                record.append(rec)
            if min_gap is not None:
                min_gap[i:i + batch] = torch.stack([g.min(-1).values for g in gp]).min(0).values.numpy()
    return out
