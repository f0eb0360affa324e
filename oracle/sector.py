"""Oracle: exact S_z = 0 sector tools for small lattices, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2 defines the energy of a trial state as the Rayleigh quotient
E(H, psi) = psi^T H psi / psi^T psi and the ground state as its minimiser.
This module builds H on the S_z = 0 sector WITHOUT the local-energy code: it
applies the Pauli operators of Sec. 4, H = (J/4) sum_<ij> (sx sx + sy sy + sz sz)
in spin-operator units, to basis bit strings with their complex phases, and
then conjugates with the Marshall sign U = prod_{i in sublattice A} sz_i
((x + y) even is sublattice A).  The Lanczos routine (full
re-orthogonalisation) gives the ground energy.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse

from .hamiltonian import bonds


def sector_states(N: int) -> np.ndarray:
    """All configurations with N/2 up spins, uint8 [C(N, N/2), N], lexicographic in the up-site sets."""
    rows = []
    for ups in itertools.combinations(range(N), N // 2):
        s = np.zeros(N, dtype=np.uint8)
        s[list(ups)] = 1
        rows.append(s)
    return np.asarray(rows, dtype=np.uint8)


def _pauli(op: str, bit: int):
    """Action of a Pauli matrix on a single spin |bit> (bit 1 = up = +1 eigenstate of sz).

    Returns (new_bit, amplitude)."""
    if op == "z":
        return bit, (1.0 if bit else -1.0)
    if op == "x":
        return 1 - bit, 1.0
    # sy |up> = i |down>, sy |down> = -i |up>
    return 1 - bit, (1j if bit else -1j)


def hamiltonian_sector(L: int, periodic: bool, J: float = 1.0):
    """Sparse (CSR) Marshall-rotated H on the S_z = 0 sector and its basis states."""
    N = L * L
    states = sector_states(N)
    index = {s.tobytes(): k for k, s in enumerate(states)}
    bl = bonds(L, periodic)
    dim = len(states)
    rows, cols, vals = [], [], []
    for k, s in enumerate(states):
        col = {}
        for (i, j) in bl:
            for op in "xyz":
                t = s.copy()
                t[i], ai = _pauli(op, int(s[i]))
                t[j], aj = _pauli(op, int(t[j]))
                # <t| sa_i sa_j |s> = ai * aj
                key = t.tobytes()
                col[key] = col.get(key, 0.0) + 0.25 * J * ai * aj
        for key, v in col.items():
            if key in index:
                rows.append(index[key])
                cols.append(k)
                vals.append(v)
            elif abs(v) > 1e-14:  # sx sx + sy sy must cancel outside the sector
                raise AssertionError("H leaks out of the S_z = 0 sector")
    vals = np.asarray(vals, dtype=np.complex128)
    if np.max(np.abs(vals.imag)) > 1e-14:
        raise AssertionError("Heisenberg matrix must be real in the S^z basis")
    H = scipy.sparse.csr_matrix((vals.real, (rows, cols)), shape=(dim, dim))  # duplicates summed
    sub_a = np.array([((p % L) + (p // L)) % 2 == 0 for p in range(N)])
    sign = np.where(states[:, sub_a].sum(axis=1) % 2 == 0, 1.0, -1.0)
    U = scipy.sparse.diags(sign)
    return (U @ H @ U).tocsr(), states


def rayleigh_quotient(H: np.ndarray, psi: np.ndarray) -> float:
    return float(psi @ (H @ psi) / (psi @ psi))


def lanczos_ground(H, iters: int = 300, seed: int = 7, tol: float = 1e-12):
    """Lowest eigenpair of symmetric H by Lanczos with full re-orthogonalisation.

    Stops when the residual ||H v - e v|| = beta_k |y_k| (y the lowest Ritz vector
    of the tridiagonal matrix) falls below ``tol``."""
    n = H.shape[0]
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    V = [v / np.linalg.norm(v)]
    alpha, beta = [], []
    for _ in range(min(iters, n)):
        w = H @ V[-1]
        alpha.append(float(V[-1] @ w))
        for u in V:  # full re-orthogonalisation (twice is enough)
            w -= (u @ w) * u
        for u in V:
            w -= (u @ w) * u
        b = float(np.linalg.norm(w))
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        evals, evecs = np.linalg.eigh(T)
        if b * abs(evecs[-1, 0]) < tol or b < 1e-14 or len(alpha) == n:
            break
        beta.append(b)
        V.append(w / b)
    vec = np.stack(V[:len(alpha)], axis=1) @ evecs[:, 0]
    vec /= np.linalg.norm(vec)
    if vec.sum() < 0:
        vec = -vec
    return float(evals[0]), vec
