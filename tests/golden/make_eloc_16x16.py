"""Writes eloc_16x16_64.txt: FP64 oracle local energies of the first 64 samples
of the 16 x 16 workload (Sec. 2 Eq. local-energy with the Sec. 3.1 network).

Workload: 16 x 16 periodic Heisenberg, J = 1; 8 layers, d_model 256, 8 heads,
codebook 256; weights ``synthetic_inputs.make_weights(256, 8, 256, 256, seed=0)``;
samples ``synthetic_inputs.make_samples(16, 64, seed=1)`` (the first 64 of any
larger batch drawn with the same seed: sample b has its own stream).

Per sample the file holds E_loc (every connected configuration recomputed in
full, float64), log psi of the sample and the smallest relative codeword gap
(l2 - l1) / l1 met in any row, layer and configuration of the sample.  Only
``oracle/`` computes these values.

    python tests/golden/make_eloc_16x16.py [n_samples]
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
from oracle import hamiltonian, model  # noqa: E402

L, LAYERS, D, HEADS, K = 16, 8, 256, 8, 256
OUT = os.path.join(HERE, "eloc_16x16_64.txt")


def main(n: int = 64) -> None:
    N = L * L
    blob = si.make_weights(N, LAYERS, D, K, seed=0)
    P = model.parse_blob(blob, N, LAYERS, D, HEADS, K)
    spins = si.make_samples(L, n, seed=1)
    rows = []
    t0 = time.time()
    for b in range(n):
        gap = np.empty(1)
        e = hamiltonian.local_energy(P, spins[b:b + 1], L, True, 1.0, min_gap=gap)[0]
        lp = model.log_psi(P, spins[b:b + 1])[0]
        rows.append((b, e, lp, gap[0]))
        print(f"{b} {e:.17g} {lp:.17g} {gap[0]:.6e}  ({time.time() - t0:.0f} s)", flush=True)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle values of the 16x16 workload (periodic Heisenberg J = 1, 8 layers,\n"
                "# d_model 256, 8 heads, codebook 256, make_weights seed 0, make_samples seed 1).\n"
                "# Written by tests/golden/make_eloc_16x16.py, which calls oracle/ only.\n"
                "# columns: sample e_loc log_psi min_relative_code_gap\n")
        for b, e, lp, g in rows:
            f.write(f"{b} {e:.17g} {lp:.17g} {g:.6e}\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 64)
