"""Writes eloc_<name>.txt for the 16 x 16 architecture-variant workloads and the
384-site Ising chain: FP64 oracle local energies of the first 16 samples of
each, with the smallest relative codeword gap met in any row, layer and
configuration of the sample.  Only ``oracle/`` computes these values.

Workloads (weights ``synthetic_inputs.make_weights(..., seed=0)`` with the
variant's blob segments; samples ``make_samples(16, 16, seed=1)`` or
``make_chain_samples(384, 16, seed=1)``):
  arch16_h1, arch16_h2, arch16_h4  16x16 periodic Heisenberg J = 1, 3 blocks,
                                   d_model 256, 8 heads, 64 codes per quantizer
                                   head, 1 / 2 / 4 quantizer heads (Table 1's
                                   6 / 12 / 24 bits)
  table1_12b                       the same with 2 quantizer heads and the final
                                   attention-only half-block (Table 1's network)
  table1_12b_g4                    table1_12b with tokens of 4 spins
  table1_48b                       Table 1's 48-bit network: 8 quantizer heads of
                                   64 codes and the final half-block
  chain384                         open transverse-field Ising chain, 384 sites,
                                   J = Gamma = 1, 1 block, d_model 256, 8 heads,
                                   64 codes (Sec. 4's largest chain)

    python tests/golden/make_eloc_variants.py [name ...]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synthetic_inputs as si  # noqa: E402
from oracle import hamiltonian, model, tfim  # noqa: E402

NS = 16
WORKLOADS = {
    # name: (L or chain sites, layers, d, heads, K, vq_heads, half_block, token_group, chain)
    "arch16_h1": (16, 3, 256, 8, 64, 1, False, 1, False),
    "arch16_h2": (16, 3, 256, 8, 64, 2, False, 1, False),
    "arch16_h4": (16, 3, 256, 8, 64, 4, False, 1, False),
    "table1_12b": (16, 3, 256, 8, 64, 2, True, 1, False),
    "table1_12b_g4": (16, 3, 256, 8, 64, 2, True, 4, False),
    "table1_48b": (16, 3, 256, 8, 64, 8, True, 1, False),
    "chain384": (384, 1, 256, 8, 64, 1, False, 1, True),
}


def run(name: str) -> None:
    L, layers, d, heads, K, H, hb, G, chain = WORKLOADS[name]
    N = L if chain else L * L
    w = si.make_weights(N, layers, d, K, seed=0, half_block=hb, token_group=G)
    P = model.parse_blob(w, N, layers, d, heads, K, vq_heads=H, half_block=hb, token_group=G)
    spins = si.make_chain_samples(N, NS, seed=1) if chain else si.make_samples(L, NS, seed=1)
    rows = []
    t0 = time.time()
    for b in range(NS):
        gap = np.empty(1)
        if chain:
            e = tfim.local_energy(P, spins[b:b + 1], periodic=False, J=1.0, Gamma=1.0, min_gap=gap)[0]
        else:
            e = hamiltonian.local_energy(P, spins[b:b + 1], L, True, 1.0, min_gap=gap)[0]
        rows.append((b, e, gap[0]))
        print(f"{name} {b} {e:.17g} {gap[0]:.6e} ({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, f"eloc_{name}.txt"), "w") as f:
        f.write(f"# FP64 oracle local energies, workload {name} (see make_eloc_variants.py for its definition).\n"
                "# Written by tests/golden/make_eloc_variants.py, which calls oracle/ only.\n"
                "# columns: sample e_loc min_relative_code_gap\n")
        for b, e, g in rows:
            f.write(f"{b} {e:.17g} {g:.6e}\n")


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(WORKLOADS)):
        run(n)
