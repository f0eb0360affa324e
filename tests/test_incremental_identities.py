"""The two identities the incremental local-energy path rests on, in FP64 numpy
(independent of the CUDA code that uses them).

1. Softmax correction.  A causal attention row whose query is unchanged but
   whose keys/values differ at a set D of earlier positions satisfies, with the
   old maximum m and normaliser l of the scaled scores,
       l' = l - sum_D e_old + sum_D e_new,
       o' = o + (sum_D e_new (v_new - o) - e_old (v_old - o)) / l',
   e_x = exp(q.k_x / sqrt(dh) - m).
2. Codeword certificate.  For the nearest codeword c of o (Eq. vq) and any
   delta, ||o+delta-W_j||^2 - ||o+delta-W_c||^2 = g_j - 2 delta.(W_j - W_c)
   with g_j the old gap; so c stays nearest whenever
   ||delta|| < (g_j) / (2 ||W_j - W_c||) for every j != c.
"""
import numpy as np


def softmax_attention(q, K, V):
    s = K @ q / np.sqrt(len(q))
    e = np.exp(s - s.max())
    return e @ V / e.sum(), s.max(), e.sum()


def test_softmax_correction_identity():
    rng = np.random.default_rng(7)
    for trial in range(200):
        dh, p = int(rng.choice([8, 16, 32])), int(rng.integers(2, 60))
        q = rng.normal(size=dh)
        K, V = rng.normal(size=(p + 1, dh)), rng.normal(size=(p + 1, dh))
        o, m, l = softmax_attention(q, K, V)
        D = rng.choice(p, size=int(rng.integers(1, min(p, 8) + 1)), replace=False)  # keys before p
        K2, V2 = K.copy(), V.copy()
        K2[D] = rng.normal(size=(len(D), dh))
        V2[D] = rng.normal(size=(len(D), dh))
        o_full, _, _ = softmax_attention(q, K2, V2)
        eo = np.exp(K[D] @ q / np.sqrt(dh) - m)
        en = np.exp(K2[D] @ q / np.sqrt(dh) - m)
        l2 = l - eo.sum() + en.sum()
        delta = (en @ (V2[D] - o) - eo @ (V[D] - o)) / l2
        assert np.allclose(o + delta, o_full, rtol=0, atol=1e-12)
        # the normaliser matches the full one in the old maximum's frame
        s2 = K2 @ q / np.sqrt(dh)
        assert np.isclose(l2, np.exp(s2 - m).sum(), rtol=1e-12)


def test_a_dropped_term_breaks_the_correction():
    """Leaving out the -(e_new - e_old) o term (the renormalisation) is caught."""
    rng = np.random.default_rng(3)
    dh, p = 16, 20
    q, K, V = rng.normal(size=dh), rng.normal(size=(p + 1, dh)), rng.normal(size=(p + 1, dh))
    o, m, l = softmax_attention(q, K, V)
    D = np.array([3, 11])
    K2, V2 = K.copy(), V.copy()
    K2[D] += 2.0
    V2[D] -= 1.0
    o_full, _, _ = softmax_attention(q, K2, V2)
    eo, en = np.exp(K[D] @ q / 4.0 - m), np.exp(K2[D] @ q / 4.0 - m)
    l2 = l - eo.sum() + en.sum()
    wrong = o + (en @ V2[D] - eo @ V[D]) / l2
    assert not np.allclose(wrong, o_full, atol=1e-6)


def test_certificate_is_sound_and_tight_per_codeword():
    rng = np.random.default_rng(11)
    kept = 0
    for trial in range(3000):
        d, K = 16, 12
        W = rng.normal(size=(K, d))
        o = rng.normal(size=d)
        dist = ((o - W) ** 2).sum(1)
        c = int(np.argmin(dist))
        wd = np.linalg.norm(W - W[c], axis=1)
        rho = np.where(np.arange(K) == c, np.inf, (dist - dist[c]) / (2 * np.where(wd > 0, wd, 1)))
        delta = rng.normal(size=d)
        delta *= rng.uniform(0, 1.5) * np.min(rho) / np.linalg.norm(delta)
        new = ((o + delta - W) ** 2).sum(1)
        # the exact gap change
        assert np.allclose(new - new[c], dist - dist[c] - 2 * (W - W[c]) @ delta, atol=1e-10)
        if np.linalg.norm(delta) < np.min(rho):
            assert int(np.argmin(new)) == c
            kept += 1
    assert kept > 500


def test_certificate_radius_is_attained():
    """Along the worst direction a step just past rho_j makes j win: the bound
    cannot be loosened."""
    rng = np.random.default_rng(5)
    d = 8
    W = rng.normal(size=(2, d))
    o = W[0] + 0.3 * (W[1] - W[0])  # nearer to W_0
    g = ((o - W[1]) ** 2).sum() - ((o - W[0]) ** 2).sum()
    u = (W[1] - W[0]) / np.linalg.norm(W[1] - W[0])
    rho = g / (2 * np.linalg.norm(W[1] - W[0]))
    for f, want in ((0.999, 0), (1.001, 1)):
        x = o + f * rho * u
        assert int(np.argmin(((x - W) ** 2).sum(1))) == want
