"""Oracle: exact autoregressive sampling of the VQ-NQS distribution, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2: psi(s) = sqrt(P(s)) with P(s) = prod_p P(s_p | s_<p), so configurations
are drawn exactly from |psi|^2 one site at a time, without Markov chains.
With the uniform numbers u[b, p] given as input (they are part of the input
here, not drawn inside), site p of sample b is up (1) when
u[b, p] < P(s_p = up | s_<p), down (0) otherwise: the inverse CDF of the
two-point conditional.  Every conditional is taken from a full forward pass of
the prefix (causal: position p of the output sees s_<p only).

With tokens of G spins (Sec. 3.1) the draw at position t is the group value v
of G spins: the smallest v with u[b, t] < sum_{w <= v} P(w | earlier groups)
(inverse CDF over the 2^G values in increasing order), whose bit k is spin
tG + k.
"""
from __future__ import annotations

import numpy as np
import torch

from . import model


def sample(P: model.Params, uniforms: np.ndarray, n_sites: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Configurations [B, N] drawn with ``uniforms`` [B, N], and P(up) of every step [B, N]."""
    u = np.asarray(uniforms, dtype=np.float64)
    B, N = u.shape
    s = np.zeros((B, N), dtype=np.int64)
    pup = np.zeros((B, N), dtype=np.float64)
    with torch.no_grad():
        for p in range(N):
            lp = model.forward(P, torch.as_tensor(s))  # [B, N, 2]; position p depends on s_<p only
            pup[:, p] = np.exp(lp[:, p, 1].numpy())
            s[:, p] = (u[:, p] < pup[:, p]).astype(np.int64)
    return s, pup


def sample_groups(P: model.Params, uniforms: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Tokens of G = P.token_group spins: configurations [B, N] drawn with ``uniforms``
    [B, N / G], and the conditionals of every step [B, N / G, 2^G]."""
    G = P.token_group
    u = np.asarray(uniforms, dtype=np.float64)
    B, T = u.shape
    N, V = T * G, 1 << G
    s = np.zeros((B, N), dtype=np.int64)
    probs = np.zeros((B, T, V), dtype=np.float64)
    with torch.no_grad():
        for t in range(T):
            lp = model.forward(P, torch.as_tensor(s))  # [B, T, V]; position t depends on earlier groups only
            probs[:, t] = np.exp(lp[:, t].numpy())
            cdf = np.cumsum(probs[:, t], axis=1)
            v = np.minimum((u[:, t:t + 1] >= cdf).sum(1), V - 1)  # the smallest v with u < cdf[v]
            for k in range(G):
                s[:, t * G + k] = (v >> k) & 1
    return s, probs
