"""Pins of the oracle's autoregressive sampler (oracle/sampler.py).

* The empirical distribution of many draws matches P(s) = psi(s)^2 computed
  from log psi over the whole basis (every count within 5 standard deviations,
  and a chi-square statistic within its 5-sigma range).
* A mutation (the two outcomes swapped) fails the same test.
* The probability recorded at each step is the model's conditional, so the sum
  of the chosen log conditionals is 2 log psi of the drawn configuration.
"""
import itertools

import numpy as np

import synthetic_inputs as si
from oracle import model, sampler

N, LAYERS, D, HEADS, K = 4, 2, 32, 4, 8


def params():
    w = si.make_weights(N, LAYERS, D, K, seed=6, std=0.3)  # larger weights: a non-uniform distribution
    return model.parse_blob(w, N, LAYERS, D, HEADS, K)


def frequencies(s):
    idx = (s * (1 << np.arange(N - 1, -1, -1))).sum(1)
    return np.bincount(idx, minlength=2 ** N) / len(s)


def exact(P):
    states = np.array(list(itertools.product([0, 1], repeat=N)))
    return np.exp(2.0 * model.log_psi(P, states))


def z_scores(freq, p, n):
    return (freq - p) / np.sqrt(np.maximum(p * (1 - p), 1e-12) / n)


def test_draws_follow_psi_squared():
    P = params()
    n = 40000
    u = si.uniforms(7, n * N).reshape(n, N)
    s, _ = sampler.sample(P, u)
    p = exact(P)
    assert abs(p.sum() - 1.0) < 1e-12
    assert p.max() / p.min() > 3.0  # the test distribution is far from uniform
    assert np.max(np.abs(z_scores(frequencies(s), p, n))) < 5.0
    chi2 = n * np.sum((frequencies(s) - p) ** 2 / p)
    dof = 2 ** N - 1
    assert abs(chi2 - dof) < 5 * np.sqrt(2 * dof)


def test_a_flipped_conditional_is_caught():
    P = params()
    n = 40000
    u = si.uniforms(8, n * N).reshape(n, N)
    s, _ = sampler.sample(P, u)
    s_bad = 1 - s  # the two outcomes swapped
    assert np.max(np.abs(z_scores(frequencies(s_bad), exact(P), n))) > 5.0


def test_recorded_conditionals_give_log_psi():
    P = params()
    u = si.uniforms(9, 64 * N).reshape(64, N)
    s, pup = sampler.sample(P, u)
    logp = np.where(s == 1, np.log(pup), np.log1p(-pup)).sum(1)
    assert np.allclose(logp, 2.0 * model.log_psi(P, s), rtol=0, atol=1e-10)


def test_group_tokens_draws_follow_psi_squared():
    """Tokens of 2 spins (16-way over 4 sites: two 4-way draws): the empirical
    distribution matches P(s) over the basis, and the recorded conditionals give
    2 log psi of the drawn configurations."""
    G = 2
    w = si.make_weights(N, LAYERS, D, K, seed=6, std=0.3, token_group=G)
    P = model.parse_blob(w, N, LAYERS, D, HEADS, K, token_group=G)
    n = 40000
    u = si.uniforms(10, n * (N // G)).reshape(n, N // G)
    s, probs = sampler.sample_groups(P, u)
    p = exact(P)
    assert abs(p.sum() - 1.0) < 1e-12 and p.max() / p.min() > 3.0
    assert np.max(np.abs(z_scores(frequencies(s), p, n))) < 5.0
    v = (s.reshape(n, N // G, G) * (1 << np.arange(G))).sum(-1)
    logp = np.log(np.take_along_axis(probs, v[..., None], -1)[..., 0]).sum(1)
    assert np.allclose(logp[:64], 2.0 * model.log_psi(P, s[:64]), rtol=0, atol=1e-10)
    # a plausible mistake, the bits of a group in the opposite order, is caught
    s_rev = s.reshape(n, N // G, G)[..., ::-1].reshape(n, N)
    assert np.max(np.abs(z_scores(frequencies(s_rev), p, n))) > 5.0
