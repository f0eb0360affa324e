"""Oracle: the one-dimensional transverse-field Ising model and its local energy, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4 defines H = -J sum_<ij> sigma^z_i sigma^z_j - Gamma sum_i sigma^x_i on a
chain (nearest neighbours, open boundaries in the paper; periodic is also
provided), studied at Gamma = 1 (the critical point).  Sec. 2 gives the row
structure for this model: the non-zero entries of row s are s itself and the N
configurations with one spin flipped.  In the sigma^z basis

  diagonal     -J sum_<ij> sigma_i sigma_j              (sigma = +1 up, -1 down)
  off-diagonal -Gamma to each s' = s with one spin flipped.

All off-diagonal elements are negative, so the ground state can be taken
positive (zero phase, as for the rotated Heisenberg model).  Local energy
(Sec. 2, Eq. local-energy):

  E_loc(s) = -J sum_<ij> sigma_i sigma_j - Gamma sum_p exp(log psi(s^p) - log psi(s)).
"""
from __future__ import annotations

import numpy as np

from . import model


def chain_bonds(N: int, periodic: bool) -> np.ndarray:
    """Nearest-neighbour bonds (p, p+1) of an N-site chain, plus (N-1, 0) when periodic (N > 2)."""
    out = [(p, p + 1) for p in range(N - 1)]
    if periodic and N > 2:
        out.append((N - 1, 0))
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


def connected(spins: np.ndarray, bond_list: np.ndarray, J: float, Gamma: float):
    """Non-zero row entries of H for one configuration: (diag, configs [N, N], h [N])."""
    s = np.asarray(spins).astype(np.int64)
    sig = 2 * s - 1
    diag = -J * float(np.sum(sig[bond_list[:, 0]] * sig[bond_list[:, 1]]))
    N = len(s)
    cfgs = np.repeat(s[None, :], N, axis=0)
    cfgs[np.arange(N), np.arange(N)] ^= 1
    return diag, cfgs, np.full(N, -Gamma)


def local_energy_fn(log_psi_fn, spins: np.ndarray, periodic: bool, J: float, Gamma: float,
                    min_gap=None) -> np.ndarray:
    """E_loc for each row of ``spins`` with an arbitrary real log-amplitude function
    (same contract as ``hamiltonian.local_energy_fn``)."""
    spins = np.asarray(spins)
    bl = chain_bonds(spins.shape[1], periodic)
    out = np.empty(spins.shape[0], dtype=np.float64)
    block = 64
    for b0 in range(0, spins.shape[0], block):
        rows, parts, start = [], [], 0
        for b in range(b0, min(b0 + block, spins.shape[0])):
            diag, cfgs, h = connected(spins[b], bl, J, Gamma)
            parts.append((b, diag, h, start, len(cfgs)))
            rows.append(np.concatenate([spins[b][None, :].astype(np.int64), cfgs], axis=0))
            start += 1 + len(cfgs)
        res = log_psi_fn(np.concatenate(rows, axis=0))
        lp, aux = (res if isinstance(res, tuple) else (res, None))
        for b, diag, h, start, n in parts:
            out[b] = diag + float(np.sum(h * np.exp(lp[start + 1:start + 1 + n] - lp[start])))
            if min_gap is not None and aux is not None:
                min_gap[b] = float(np.min(aux[start:start + 1 + n]))
    return out


def local_energy(P: model.Params, spins: np.ndarray, periodic: bool = False, J: float = 1.0, Gamma: float = 1.0,
                 batch: int = 64, min_gap=None) -> np.ndarray:
    """E_loc(s) of the VQ-NQS wave function for the chain, every flipped configuration recomputed in full."""
    def fn(c):
        if min_gap is None:
            return model.log_psi(P, c, batch=batch)
        g = np.empty(len(c))
        return model.log_psi(P, c, batch=batch, min_gap=g), g
    return local_energy_fn(fn, spins, periodic, J, Gamma, min_gap=min_gap)
