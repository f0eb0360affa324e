"""Oracle: square-lattice Heisenberg bonds and the local energy, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4 defines H = sum_<ij> sigma_i . sigma_j on nearest neighbours.  The
energies the paper prints (Table 1, 4x4: -0.574325 per site) are those of the
spin operators S = sigma / 2, so the oracle uses H = J sum_<ij> S_i . S_j.
In the S^z basis rotated by the Marshall sign rule (Sec. 4: the ground state
is then positive, the phase is zero) a bond contributes

  diagonal     (J/4) sigma_i sigma_j        (sigma = +1 up, -1 down)
  off-diagonal -J/2 to s' = s with spins i and j exchanged, when s_i != s_j.

Local energy (Sec. 2, Eq. local-energy):

  E_loc(s) = sum_s' H_{s s'} psi(s') / psi(s)
           = (J/4) sum_b sigma_i sigma_j - (J/2) sum_{b: s_i != s_j} exp(log psi(s^b) - log psi(s)).

Bonds: site p = y L + x links to ((x+1) mod L, y) and (x, (y+1) mod L) when
periodic; open boundaries drop the wrapped links.  With periodic L = 2 both
links of a pair appear, so every pair is counted twice (kept on purpose: it is
what the 2N-bond rule gives).
"""
from __future__ import annotations

import numpy as np

from . import model


def bonds(L: int, periodic: bool) -> np.ndarray:
    """Nearest-neighbour bonds as an int array [n_b, 2] of raster site indices."""
    out = []
    for y in range(L):
        for x in range(L):
            p = y * L + x
            if x + 1 < L or periodic:
                out.append((p, y * L + (x + 1) % L))
            if y + 1 < L or periodic:
                out.append((p, ((y + 1) % L) * L + x))
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


def connected(spins: np.ndarray, bond_list: np.ndarray, J: float):
    """Non-zero row entries of H for one configuration.

    Returns (diag, configs, h): the diagonal element and the off-diagonal
    configurations s' with their matrix elements H_{s s'} (all -J/2)."""
    s = np.asarray(spins).astype(np.int64)
    sig = 2 * s - 1
    i, j = bond_list[:, 0], bond_list[:, 1]
    diag = 0.25 * J * float(np.sum(sig[i] * sig[j]))
    anti = np.nonzero(s[i] != s[j])[0]
    cfgs = np.repeat(s[None, :], len(anti), axis=0)
    for r, b in enumerate(anti):
        a, c = bond_list[b]
        cfgs[r, a], cfgs[r, c] = s[c], s[a]
    return diag, cfgs, np.full(len(anti), -0.5 * J)


def local_energy_fn(log_psi_fn, spins: np.ndarray, L: int, periodic: bool, J: float, min_gap=None) -> np.ndarray:
    """E_loc for each row of ``spins`` with an arbitrary real log-amplitude function.

    ``log_psi_fn`` maps an int array [C, N] to float64 [C], or to a pair
    (log psi [C], diagnostic [C]); with ``min_gap`` given, the per-sample minimum
    of the diagnostic over the sample's configurations is stored there."""
    bl = bonds(L, periodic)
    spins = np.asarray(spins)
    out = np.empty(spins.shape[0], dtype=np.float64)
    # log psi of many samples' configurations is evaluated in one call; each
    # value still comes from its own full forward pass.
    block = 256
    for b0 in range(0, spins.shape[0], block):
        rows, parts, start = [], [], 0
        for b in range(b0, min(b0 + block, spins.shape[0])):
            diag, cfgs, h = connected(spins[b], bl, J)
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


def local_energy(P: model.Params, spins: np.ndarray, L: int, periodic: bool, J: float = 1.0,
                 batch: int = 64, min_gap=None) -> np.ndarray:
    """E_loc(s) of the VQ-NQS wave function, every connected configuration recomputed in full.

    ``min_gap`` (float64 array of len(spins)) receives per sample the smallest
    relative codeword gap met in any of its configurations (a diagnostic)."""
    def fn(c):
        if min_gap is None:
            return model.log_psi(P, c, batch=batch)
        g = np.empty(len(c))
        return model.log_psi(P, c, batch=batch, min_gap=g), g
    return local_energy_fn(fn, spins, L, periodic, J, min_gap=min_gap)
