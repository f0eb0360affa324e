"""Oracle: straight-through O_k = d log psi / d theta and the VMC energy gradient, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.1, Eq. st: the quantizer output is rewritten as V = g(D)^T W with
D_j = -||o - W_j||_2 and

  g(z) = SG[onehot(argmax_j z_j)] + softmax(z) - SG[softmax(z)],

so the forward value is the nearest codeword and the backward pass flows
through softmax(D) (straight-through, temperature 1, no noise: the paper's
"variant of Gumbel-Softmax" is read as this noiseless form).  With H quantizer
heads the expression is applied per head, V_h = g(D_h)^T W_h, as Eq. st is
written.  The gradient is taken by torch autograd on exactly that expression.

Sec. 2 gradient estimator: dE/dtheta ~ sum_i (E_loc(s_i) - E)^* d log Psi(s_i)/dtheta.
Read with the 1/B normalisation and the factor 2 that the derivative of the
Rayleigh quotient carries for a real wave function:

  grad_E = 2 * mean_s[(E_loc(s) - mean E_loc) * O(s)].

The flat gradient vector follows the weight-blob order (including the unused
rows of pos_emb, whose entries are zero).
"""
from __future__ import annotations

import numpy as np
import torch

from . import model


def _leaf_params(P: model.Params) -> model.Params:
    t = {k: v.detach().clone().requires_grad_(True) for k, v in P.t.items()}
    return model.Params(d=P.d, heads=P.heads, K=P.K, layers=P.layers, n_max=P.n_max, t=t, vq_heads=P.vq_heads,
                        half_block=P.half_block, token_group=P.token_group)


def _heads(W, o):
    """(segments of o, codebooks): one pair per quantizer head (one for a [K, d] codebook)."""
    if W.dim() == 2:
        return [o], [W]
    H, K, dq = W.shape
    return [o[..., h * dq:(h + 1) * dq] for h in range(H)], [W[h] for h in range(H)]


def _soft_D(seg, Wh):
    """softmax over j of D_j = -||seg - W_h,j||_2."""
    D = -torch.sqrt(torch.clamp(((seg[..., None, :] - Wh) ** 2).sum(-1), min=0.0))
    return torch.softmax(D, dim=-1)


def st_quantizer(P: model.Params):
    """Eq. st with SG = detach, per quantizer head."""
    def q(l, o):
        parts, codes = [], []
        for seg, Wh in zip(*_heads(P.t[f"{l}.codebook"], o)):
            c = torch.argmin(model.sq_distances(seg, Wh), dim=-1)
            soft = _soft_D(seg, Wh)
            onehot = torch.nn.functional.one_hot(c, Wh.shape[0]).to(o.dtype)
            parts.append((onehot.detach() + soft - soft.detach()) @ Wh)
            codes.append(c)
        return torch.cat(parts, dim=-1), codes[0] if len(codes) == 1 else torch.stack(codes, -1)
    return q


def frozen_quantizer(P: model.Params, frozen):
    """The straight-through surrogate with every stop-gradient term frozen at theta_0.

    ``frozen[l] = [(codes, softmax(D_0)) per head]``.  Its value is
    onehot(c_0)^T W + (softmax(D(theta)) - softmax(D_0))^T W per head, whose
    derivative at theta_0 equals the straight-through gradient; finite
    differences of it check Eq. st."""
    def q(l, o):
        parts, codes = [], []
        for (seg, Wh), (c0, soft0) in zip(zip(*_heads(P.t[f"{l}.codebook"], o)), frozen[l]):
            onehot = torch.nn.functional.one_hot(c0, Wh.shape[0]).to(o.dtype)
            parts.append((onehot + _soft_D(seg, Wh) - soft0) @ Wh)
            codes.append(c0)
        return torch.cat(parts, dim=-1), codes[0] if len(codes) == 1 else torch.stack(codes, -1)
    return q


def record_frozen(P: model.Params, spins):
    """Codes and softmax(D) of every layer and head at the current parameters, for ``frozen_quantizer``."""
    frozen = []

    def q(l, o):
        per_head, parts = [], []
        for seg, Wh in zip(*_heads(P.t[f"{l}.codebook"], o)):
            c = model.nearest_code(seg, Wh)
            per_head.append((c, _soft_D(seg, Wh)))
            parts.append(Wh[c])
        frozen.append(per_head)
        return torch.cat(parts, dim=-1), per_head[0][0]

    with torch.no_grad():
        model.forward(P, spins, quantizer=q)
    return frozen


def log_psi_with(P: model.Params, spins, quantizer) -> torch.Tensor:
    s = torch.as_tensor(np.asarray(spins)).long()
    lp = model.forward(P, s, quantizer=quantizer)
    v = model.group_values(s, P.token_group)
    return 0.5 * lp.gather(-1, v[..., None])[..., 0].sum(-1)


def flatten(P: model.Params, grads: dict) -> np.ndarray:
    out = []
    for name in P.t:  # insertion order == blob order
        g = grads.get(name)
        out.append(np.zeros(P.t[name].numel()) if g is None else g.detach().reshape(-1).numpy())
    return np.concatenate(out)


def per_sample_O(P: model.Params, spins) -> np.ndarray:
    """O[b, k] = d log psi(s_b) / d theta_k through the straight-through quantizer."""
    spins = np.asarray(spins)
    Q = _leaf_params(P)
    names = list(Q.t)
    out = []
    for b in range(spins.shape[0]):
        lp = log_psi_with(Q, spins[b:b + 1], st_quantizer(Q))[0]
        gs = torch.autograd.grad(lp, [Q.t[n] for n in names], allow_unused=True)
        out.append(flatten(Q, dict(zip(names, gs))))
    return np.stack(out)


def energy_gradient(O: np.ndarray, e_loc: np.ndarray, weights=None) -> np.ndarray:
    """grad_E = 2 mean_s[(E_loc(s) - mean E_loc) O(s)].

    With ``weights`` (e.g. |psi|^2 over a whole sector) the means are the
    weighted ones, which turns the estimator into the exact derivative of the
    Rayleigh quotient."""
    e = np.asarray(e_loc, dtype=np.float64)
    w = np.ones_like(e) if weights is None else np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    ebar = float(np.sum(w * e))
    return 2.0 * ((w * (e - ebar))[:, None] * O).sum(axis=0)
