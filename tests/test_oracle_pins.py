"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a
printed value, a closed form, an exact identity, a library routine or brute
force, chosen so that a dropped term, a wrong sign or a transposed operand in
the oracle fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse.linalg
import torch

import synthetic_inputs as si
from conftest import read_golden
from oracle import gradient, hamiltonian, model, sector

pytestmark = pytest.mark.filterwarnings("ignore::UserWarning")


def small_model(N, layers=2, d=16, heads=4, K=8, seed=3, std=0.2):
    blob = si.make_weights(N, layers, d, K, seed=seed, std=std)
    return blob, model.parse_blob(blob, N, layers, d, heads, K)


# --- lattice and Hamiltonian (Sec. 2 k-local H, Sec. 4 Heisenberg) -----------

@pytest.mark.parametrize("L", [2, 3, 4, 5, 6, 16])
def test_bond_counts(L):
    assert len(hamiltonian.bonds(L, True)) == 2 * L * L
    assert len(hamiltonian.bonds(L, False)) == 2 * L * (L - 1)
    # every open bond joins nearest neighbours
    for i, j in hamiltonian.bonds(L, False):
        (yi, xi), (yj, xj) = divmod(int(i), L), divmod(int(j), L)
        assert abs(xi - xj) + abs(yi - yj) == 1


def test_sector_size():
    assert len(sector.sector_states(16)) == math.comb(16, 8)
    assert np.all(sector.sector_states(16).sum(1) == 8)


@pytest.mark.parametrize("L,periodic,e0", [(2, True, -4.0), (2, False, -2.0)])
def test_lanczos_closed_form_2x2(L, periodic, e0):
    # 2x2 open: a 4-site ring, E0 = -2J (S=0 of S_A . S_B with S_A = S_B = 1);
    # 2x2 periodic doubles every bond, E0 = -4J.
    H, _ = sector.hamiltonian_sector(L, periodic)
    e, v = sector.lanczos_ground(H)
    assert abs(e - e0) < 1e-12
    assert np.all(v > 0)  # Marshall-rotated ground state is positive


def test_lanczos_4x4_open_matches_table1():
    g = read_golden("heisenberg_4x4_open_e0.txt")
    H, _ = sector.hamiltonian_sector(int(g["L"]), bool(int(g["periodic"])))
    e, v = sector.lanczos_ground(H)
    assert abs(e / 16 - float(g["e0_per_site"])) <= float(g["tolerance"])
    # and against a library eigensolver
    ref = scipy.sparse.linalg.eigsh(H, k=1, which="SA")[0][0]
    assert abs(e - ref) < 1e-9
    assert np.all(v > 0)


def test_hamiltonian_symmetric():
    H, _ = sector.hamiltonian_sector(4, True)
    assert abs(H - H.T).max() == 0.0


# --- local energy (Sec. 2, Eq. local-energy) ----------------------------------

@pytest.mark.parametrize("L,periodic", [(2, True), (2, False), (4, True)])
def test_local_energy_rayleigh_identity(L, periodic):
    """sum |psi|^2 E_loc / sum |psi|^2 == psi^T H psi / psi^T psi on the whole sector,
    with H built from the Pauli form independently of the E_loc code."""
    N = L * L
    _, P = small_model(N)
    H, states = sector.hamiltonian_sector(L, periodic)
    lp = model.log_psi(P, states, batch=4096)
    el = hamiltonian.local_energy(P, states, L, periodic, 1.0, batch=4096)
    psi = np.exp(lp)
    w = psi ** 2
    rq = sector.rayleigh_quotient(H, psi)
    assert abs(np.sum(w * el) / np.sum(w) - rq) < 1e-10
    e0, _ = sector.lanczos_ground(H)
    assert rq >= e0 - 1e-10  # variational bound


def test_local_energy_zero_variance_on_ground_state():
    """With psi the exact ground state, E_loc(s) = E0 for every s."""
    L = 4
    H, states = sector.hamiltonian_sector(L, False)
    e0, v = sector.lanczos_ground(H, tol=1e-12, iters=400)
    assert np.linalg.norm(H @ v - e0 * v) < 1e-10
    index = {s.tobytes(): k for k, s in enumerate(states)}

    def lp_fn(cfgs):
        return np.log(np.array([v[index[c.astype(np.uint8).tobytes()]] for c in cfgs]))

    el = hamiltonian.local_energy_fn(lp_fn, states[::97], L, False, 1.0)
    assert np.max(np.abs(el - e0)) < 1e-8


def test_local_energy_uniform_amplitude_closed_form():
    """All weights zero except the head bias: log psi depends only on the number of
    up spins, exchanges keep it, every ratio is 1 and
    E_loc = (J/4) sum_b sigma_i sigma_j - (J/2) * #anti-aligned bonds."""
    L, N, layers, d, K = 4, 16, 2, 8, 4
    blob = np.zeros(si.num_params(N, layers, d, K), dtype=np.float32)
    P = model.parse_blob(blob, N, layers, d, 2, K)
    for k in P.t:
        if k.endswith("_g"):
            P.t[k][:] = 1.0
    P.t["b_head"][:] = torch.tensor([0.3, -0.8], dtype=torch.float64)
    spins = si.make_samples(L, 8, seed=5)
    lsm = torch.log_softmax(P.t["b_head"], 0).numpy()
    want_lp = 0.5 * np.array([lsm[s].sum() for s in spins])
    assert np.allclose(model.log_psi(P, spins), want_lp, atol=1e-13)
    J = 1.7
    bl = hamiltonian.bonds(L, True)
    sig = 2 * spins.astype(np.int64) - 1
    want = 0.25 * J * (sig[:, bl[:, 0]] * sig[:, bl[:, 1]]).sum(1) \
        - 0.5 * J * (spins[:, bl[:, 0]] != spins[:, bl[:, 1]]).sum(1)
    assert np.allclose(hamiltonian.local_energy(P, spins, L, True, J), want, atol=1e-12)


# --- the wave function (Sec. 2 chain rule, Sec. 3.1) --------------------------

@pytest.mark.parametrize("N", [4, 8])
def test_autoregressive_normalisation(N):
    """P(s) = prod_p P(s_p | s_<p) sums to one over all 2^N configurations; fails if
    the causal mask leaks the future or the input is not shifted right."""
    _, P = small_model(N, std=0.5)
    allc = np.array(list(itertools.product([0, 1], repeat=N)))
    assert abs(np.exp(2 * model.log_psi(P, allc)).sum() - 1.0) < 1e-12


def test_causality():
    N = 9
    _, P = small_model(N, std=0.5)
    s = np.array([[1, 0, 0, 1, 1, 0, 1, 0, 0]])
    for j in range(N):
        t = s.copy()
        t[0, j] ^= 1
        a = model.forward(P, torch.as_tensor(s))
        b = model.forward(P, torch.as_tensor(t))
        # conditionals of positions <= j see only s_<p, which is unchanged
        assert torch.equal(a[0, :j + 1], b[0, :j + 1])
        if j + 1 < N:
            assert not torch.allclose(a[0, j + 1:], b[0, j + 1:])


def test_single_codeword_makes_attention_irrelevant():
    """With one codeword the quantizer output is constant, so the attention weights
    cannot change log psi."""
    N = 9
    blob, P = small_model(N, K=1, std=0.5)
    s = np.array([[1, 0, 1, 1, 0, 0, 1, 0, 1]])
    a = model.log_psi(P, s)
    for l in range(P.layers):
        P.t[f"{l}.w_qkv"] = torch.randn_like(P.t[f"{l}.w_qkv"])
    assert np.array_equal(a, model.log_psi(P, s))


def test_nearest_code_brute_force_and_ties():
    rng = np.random.default_rng(0)
    for _ in range(20):
        o = rng.standard_normal((7, 5))
        W = rng.standard_normal((11, 5))
        got = model.nearest_code(torch.as_tensor(o), torch.as_tensor(W)).numpy()
        for r in range(7):
            dist = [sum((o[r, t] - W[j, t]) ** 2 for t in range(5)) for j in range(11)]
            assert got[r] == int(np.argmin(dist))
    # exact ties go to the lowest index
    W = torch.tensor([[0.0, 2.0], [1.0, 0.0], [-1.0, 0.0], [0.0, -2.0], [1.0, 0.0]], dtype=torch.float64)
    o = torch.zeros(1, 2, dtype=torch.float64)
    assert model.nearest_code(o, W).item() == 1
    o = torch.tensor([[1.0, 0.0]], dtype=torch.float64)
    assert model.nearest_code(o, W).item() == 1
    o = torch.tensor([[0.0, 0.0]], dtype=torch.float64)
    assert model.nearest_code(o, W[[3, 0, 2, 1]]).item() == 2


def test_attention_matches_library_sdpa():
    rng = np.random.default_rng(1)
    C, N, d, h = 3, 7, 12, 3
    a = torch.as_tensor(rng.standard_normal((C, N, d)))
    w = torch.as_tensor(rng.standard_normal((d, 3 * d)) * 0.4)
    b = torch.as_tensor(rng.standard_normal(3 * d) * 0.1)
    got = model.causal_attention(a, w, b, h)
    qkv = a @ w + b
    q, k, v = (qkv[..., i * d:(i + 1) * d].reshape(C, N, h, d // h).transpose(1, 2) for i in range(3))
    ref = torch.nn.functional.scaled_dot_product_attention(q, k, v, is_causal=True)
    assert torch.allclose(got, ref.transpose(1, 2).reshape(C, N, d), atol=1e-13)


def test_forward_matches_torch_nn_composition():
    """The same network assembled from torch.nn library modules (MultiheadAttention,
    LayerNorm, Linear, erf-GELU) with the blob's weights loaded into them."""
    N, layers, d, heads, K = 10, 2, 16, 4, 8
    # every entry random, biases and LayerNorm gains/shifts included
    blob = (si.make_weights(N, layers, d, K, seed=3, std=0.4)
            + 0.3 * si.normals(11, si.num_params(N, layers, d, K))).astype(np.float32)
    P = model.parse_blob(blob, N, layers, d, heads, K)
    blob = np.asarray(blob, dtype=np.float64)
    torch.manual_seed(0)
    spins = torch.as_tensor(np.array([[1, 0, 0, 1, 1, 0, 1, 0, 0, 1], [0, 1, 1, 0, 0, 1, 1, 0, 1, 0]]))
    pos = 0

    def take(*shape):
        nonlocal pos
        n = int(np.prod(shape))
        out = torch.as_tensor(blob[pos:pos + n].reshape(shape))
        pos += n
        return out

    tok, pe = take(3, d), take(N, d)
    tokens = torch.cat([torch.full((2, 1), 2), spins[:, :-1]], 1)
    x = tok[tokens] + pe[:N]
    mask = torch.nn.Transformer.generate_square_subsequent_mask(N, dtype=torch.float64)
    for _ in range(layers):
        ln1 = torch.nn.LayerNorm(d, eps=1e-5).double()
        ln1.weight.data, ln1.bias.data = take(d), take(d)
        mha = torch.nn.MultiheadAttention(d, heads, batch_first=True).double()
        mha.in_proj_weight.data, mha.in_proj_bias.data = take(d, 3 * d).T.contiguous(), take(3 * d)
        mha.out_proj.weight.data = torch.eye(d, dtype=torch.float64)
        mha.out_proj.bias.data = torch.zeros(d, dtype=torch.float64)
        cb = take(K, d)
        wo = torch.nn.Linear(d, d).double()
        wo.weight.data, wo.bias.data = take(d, d).T.contiguous(), take(d)
        ln2 = torch.nn.LayerNorm(d, eps=1e-5).double()
        ln2.weight.data, ln2.bias.data = take(d), take(d)
        f1 = torch.nn.Linear(d, 4 * d).double()
        f1.weight.data, f1.bias.data = take(d, 4 * d).T.contiguous(), take(4 * d)
        f2 = torch.nn.Linear(4 * d, d).double()
        f2.weight.data, f2.bias.data = take(4 * d, d).T.contiguous(), take(d)
        a = ln1(x)
        o, _ = mha(a, a, a, attn_mask=mask, need_weights=False)
        code = torch.cdist(o, cb.expand(2, K, d)).argmin(-1)
        y = x + wo(cb[code])
        x = y + f2(torch.nn.functional.gelu(f1(ln2(y)), approximate="none"))
    lnf = torch.nn.LayerNorm(d, eps=1e-5).double()
    lnf.weight.data, lnf.bias.data = take(d), take(d)
    head = torch.nn.Linear(d, 2).double()
    head.weight.data, head.bias.data = take(d, 2).T.contiguous(), take(2)
    assert pos == len(blob)
    ref = torch.log_softmax(head(lnf(x)), -1)
    got = model.forward(P, spins)
    assert torch.allclose(got, ref, atol=1e-12)


# --- gradient (Sec. 2 estimator, Sec. 3.1 Eq. st) ------------------------------

def test_st_gradient_matches_finite_differences_of_surrogate():
    """Central differences (h = 1e-6) of the straight-through surrogate, with the
    stop-gradient terms frozen at theta_0, equal the autograd O_k."""
    L, N = 4, 16
    blob, P = small_model(N, layers=2, d=16, heads=4, K=8, std=0.3)
    s = si.make_samples(L, 1, seed=9)
    O = gradient.per_sample_O(P, s)[0]
    frozen = gradient.record_frozen(P, s)
    names = list(P.t)
    sizes = [P.t[n].numel() for n in names]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(4)
    picks = list(rng.choice(len(O), 150, replace=False))
    for n in ("0.codebook", "1.codebook", "b_head", "lnf_g"):
        k = names.index(n)
        picks += list(range(offs[k], min(offs[k] + 8, offs[k + 1])))
    h = 1e-6
    for g in picks:
        k = int(np.searchsorted(offs, g, side="right") - 1)
        name, j = names[k], int(g - offs[k])
        vals = []
        for sgn in (+1, -1):
            Q = model.Params(P.d, P.heads, P.K, P.layers, P.n_max, {a: b.clone() for a, b in P.t.items()})
            Q.t[name].view(-1)[j] += sgn * h
            with torch.no_grad():
                vals.append(float(gradient.log_psi_with(Q, s, gradient.frozen_quantizer(Q, frozen))[0]))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - O[g]) <= 1e-7 * max(1.0, abs(O[g])), (name, j, fd, O[g])


def test_energy_gradient_is_rayleigh_derivative_with_one_codeword():
    """With K = 1 the quantizer is constant, the straight-through gradient is the true
    gradient, and the |psi|^2-weighted estimator over the whole sector equals the
    finite-difference derivative of psi^T H psi / psi^T psi."""
    L, N = 2, 4
    blob, P = small_model(N, layers=1, d=8, heads=2, K=1, std=0.5)
    H, states = sector.hamiltonian_sector(L, False)
    lp = model.log_psi(P, states)
    el = hamiltonian.local_energy(P, states, L, False, 1.0)
    O = gradient.per_sample_O(P, states)
    g = gradient.energy_gradient(O, el, weights=np.exp(2 * lp))
    names = list(P.t)
    offs = np.concatenate([[0], np.cumsum([P.t[n].numel() for n in names])])
    rng = np.random.default_rng(2)
    h = 1e-6
    for gi in rng.choice(len(g), 60, replace=False):
        k = int(np.searchsorted(offs, gi, side="right") - 1)
        vals = []
        for sgn in (+1, -1):
            Q = model.Params(P.d, P.heads, P.K, P.layers, P.n_max, {a: b.clone() for a, b in P.t.items()})
            Q.t[names[k]].view(-1)[int(gi - offs[k])] += sgn * h
            vals.append(sector.rayleigh_quotient(H, np.exp(model.log_psi(Q, states))))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[gi]) <= 1e-7 * max(1.0, abs(g[gi])), (names[k], fd, g[gi])


def test_generators_are_deterministic_and_balanced():
    a = si.make_samples(16, 4, seed=1)
    b = si.make_samples(16, 4, seed=1)
    assert np.array_equal(a, b) and np.all(a.sum(1) == 128)
    z = si.normals(0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    w = si.make_weights(16, 2, 32, 16)
    assert w.dtype == np.float32 and len(w) == si.num_params(16, 2, 32, 16)
