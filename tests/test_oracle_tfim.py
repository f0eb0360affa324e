"""Pins of the chain transverse-field Ising oracle (oracle/tfim.py).

* The Hamiltonian it implies (diagonal + flipped rows) equals the one built
  independently from Kronecker products of Pauli matrices, entry by entry.
* The exact ground state (dense eigensolver) gives E_loc(s) = E0 for every
  configuration (zero variance of the local energy at an eigenstate).
* Closed forms: Gamma = 0 (classical chain, E_loc of the aligned state is
  -J * bonds) and J = 0 (free spins: the uniform state is exact, E_loc = -Gamma N).
* E_loc of the VQ-NQS model equals (H psi)(s) / psi(s) evaluated with the
  dense Hamiltonian and the model's amplitudes over the whole basis.
"""
import itertools

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import model, tfim

SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SZ = np.array([[1.0, 0.0], [0.0, -1.0]])  # basis order (up, down): up has sigma = +1


def basis(N):
    """All configurations, row r = bits of r with site 0 most significant; spin 1 = up.
    Kronecker index of a configuration: up maps to index 0 of each factor."""
    return np.array(list(itertools.product([1, 0], repeat=N)), dtype=np.int64)


def op_at(M, p, N):
    out = np.eye(1)
    for q in range(N):
        out = np.kron(out, M if q == p else np.eye(2))
    return out


def dense_h(N, periodic, J, G):
    H = np.zeros((2 ** N, 2 ** N))
    for a, b in tfim.chain_bonds(N, periodic):
        H -= J * op_at(SZ, a, N) @ op_at(SZ, b, N)
    for p in range(N):
        H -= G * op_at(SX, p, N)
    return H


@pytest.mark.parametrize("N,periodic", [(4, False), (5, True), (6, False), (6, True)])
def test_rows_match_kronecker_hamiltonian(N, periodic):
    J, G = 0.7, 1.3
    H = dense_h(N, periodic, J, G)
    states = basis(N)
    index = {tuple(s): i for i, s in enumerate(states)}
    Ho = np.zeros_like(H)
    bl = tfim.chain_bonds(N, periodic)
    for i, s in enumerate(states):
        diag, cfgs, h = tfim.connected(s, bl, J, G)
        Ho[i, i] += diag
        for c, v in zip(cfgs, h):
            Ho[i, index[tuple(c)]] += v
    assert np.allclose(Ho, H, rtol=0, atol=1e-12)  # equal up to summation order


@pytest.mark.parametrize("N,periodic", [(6, False), (8, True), (8, False)])
def test_exact_ground_state_has_constant_local_energy(N, periodic):
    J, G = 1.0, 1.0
    H = dense_h(N, periodic, J, G)
    w, V = np.linalg.eigh(H)
    psi = np.abs(V[:, 0])  # positive ground state (all off-diagonal entries <= 0)
    states = basis(N)
    index = {tuple(s): i for i, s in enumerate(states)}
    logpsi = lambda c: np.log(psi[[index[tuple(r)] for r in c]])
    e = tfim.local_energy_fn(logpsi, states, periodic, J, G)
    assert np.allclose(e, w[0], rtol=0, atol=1e-9)


def test_closed_forms():
    N = 7
    up = np.ones((1, N), dtype=np.int64)
    flat = lambda c: np.zeros(len(c))
    # Gamma = 0: an aligned state, no off-diagonal term
    assert tfim.local_energy_fn(flat, up, False, 1.5, 0.0)[0] == pytest.approx(-1.5 * (N - 1))
    assert tfim.local_energy_fn(flat, up, True, 1.5, 0.0)[0] == pytest.approx(-1.5 * N)
    # J = 0: the uniform state is the ground state of -Gamma sum sigma^x, E_loc = -Gamma N everywhere
    s = si.make_chain_samples(N, 5, seed=3).astype(np.int64)
    assert np.allclose(tfim.local_energy_fn(flat, s, False, 0.0, 0.8), -0.8 * N)


def test_model_local_energy_is_h_psi_over_psi():
    N, layers, d, heads, K = 6, 2, 32, 4, 8
    P = model.parse_blob(si.make_weights(N, layers, d, K, seed=4), N, layers, d, heads, K)
    states = basis(N)
    lp = model.log_psi(P, states)
    psi = np.exp(lp)
    H = dense_h(N, False, 1.0, 1.0)
    want = (H @ psi) / psi
    got = tfim.local_energy(P, states, periodic=False, J=1.0, Gamma=1.0)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_a_wrong_sign_is_caught():
    """Mutation check: flipping the sign of the transverse field breaks the composition pin."""
    N = 5
    states = basis(N)
    H = dense_h(N, False, 1.0, 1.0)
    psi = np.exp(0.1 * np.arange(len(states)) % 1.0)
    index = {tuple(s): i for i, s in enumerate(states)}
    logpsi = lambda c: np.log(psi[[index[tuple(r)] for r in c]])
    good = tfim.local_energy_fn(logpsi, states, False, 1.0, 1.0)
    bad = tfim.local_energy_fn(logpsi, states, False, 1.0, -1.0)
    want = (H @ psi) / psi
    assert np.allclose(good, want) and not np.allclose(bad, want)
