"""Oracle: straight-through O_k = d log psi / d theta and the VMC energy gradient, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.1, Eq. st: the quantizer output is rewritten as V = g(D)^T W with
D_j = -||o - W_j||_2 and

  g(z) = SG[onehot(argmax_j z_j)] + softmax(z) - SG[softmax(z)],

so the forward value is the nearest codeword and the backward pass flows
through softmax(D) (straight-through, temperature 1, no noise: the paper's
"variant of Gumbel-Softmax" is read as this noiseless form).  The gradient is
taken by torch autograd on exactly that expression.

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
    return model.Params(d=P.d, heads=P.heads, K=P.K, layers=P.layers, n_max=P.n_max, t=t)


def st_quantizer(P: model.Params):
    """Eq. st with SG = detach."""
    def q(l, o):
        W = P.t[f"{l}.codebook"]
        dist2 = model.sq_distances(o, W)
        c = torch.argmin(dist2, dim=-1)
        D = -torch.sqrt(torch.clamp(((o[..., None, :] - W) ** 2).sum(-1), min=0.0))
        soft = torch.softmax(D, dim=-1)
        onehot = torch.nn.functional.one_hot(c, W.shape[0]).to(o.dtype)
        g = onehot.detach() + soft - soft.detach()
        return g @ W, c
    return q


def frozen_quantizer(P: model.Params, frozen):
    """The straight-through surrogate with every stop-gradient term frozen at theta_0.

    ``frozen[l] = (codes, softmax(D_0))``.  Its value is onehot(c_0)^T W +
    (softmax(D(theta)) - softmax(D_0))^T W, whose derivative at theta_0 equals
    the straight-through gradient; finite differences of it check Eq. st."""
    def q(l, o):
        W = P.t[f"{l}.codebook"]
        c0, soft0 = frozen[l]
        D = -torch.sqrt(torch.clamp(((o[..., None, :] - W) ** 2).sum(-1), min=0.0))
        soft = torch.softmax(D, dim=-1)
        onehot = torch.nn.functional.one_hot(c0, W.shape[0]).to(o.dtype)
        return (onehot + soft - soft0) @ W, c0
    return q


def record_frozen(P: model.Params, spins):
    """Codes and softmax(D) of every layer at the current parameters, for ``frozen_quantizer``."""
    frozen = []

    def q(l, o):
        W = P.t[f"{l}.codebook"]
        c = model.nearest_code(o, W)
        D = -torch.sqrt(torch.clamp(((o[..., None, :] - W) ** 2).sum(-1), min=0.0))
        frozen.append((c, torch.softmax(D, dim=-1)))
        return W[c], c

    with torch.no_grad():
        model.forward(P, spins, quantizer=q)
    return frozen


def log_psi_with(P: model.Params, spins, quantizer) -> torch.Tensor:
    s = torch.as_tensor(np.asarray(spins)).long()
    lp = model.forward(P, s, quantizer=quantizer)
    return 0.5 * lp.gather(-1, s[..., None])[..., 0].sum(-1)


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
