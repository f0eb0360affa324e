"""FP64 CPU oracle for the VQ-NQS local-energy path (arXiv 2212.11296).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from here.  The product
path (``paper_2212_11296_gb300``) never imports it and shares no code with it;
the only common input is the seeded generator module ``synthetic_inputs``.

Everything here is the plain definition, evaluated in float64 with torch CPU
ops as the linear-algebra library: every connected configuration is
recomputed in full (no deduplication, no prefix reuse).

Modules:
  model        the autoregressive VQ transformer  log psi  (Sec. 3.1, Eq. vq)
  hamiltonian  bonds and the local energy  (Sec. 2 Eq. local-energy, Sec. 4)
  tfim         the chain transverse-field Ising model's local energy (Sec. 2, Sec. 4)
  sampler      exact autoregressive sampling with given uniforms (Sec. 2)
  sector       S_z = 0 sector, independently built H, Rayleigh quotient,
               Lanczos  (Sec. 2 Rayleigh quotient)
  gradient     straight-through O_k and the VMC energy gradient
               (Sec. 2 gradient estimator, Sec. 3.1 Eq. st)

Parity status: the forward pass has no printed value in the paper; it is
pinned by invariants (autoregressive normalisation, causality, a composition of
library modules, closed forms) rather than by a worked example.
"""
from . import model, hamiltonian, sector, gradient, sampler, tfim  # noqa: F401
