"""The one exchange step of a sample-sharded VMC gradient (Sec. 2 gradient estimator).

Samples are independent units: each rank (one GPU) evaluates its own samples'
local energies and log-psi gradients.  The energy gradient
grad_k = 2 mean[(E - mean E) O_k] over all ranks' samples needs the global mean
energy, which is only known after an exchange; with
sum_b (E_b - Ebar) O_b = sum_b E_b O_b - Ebar sum_b O_b, one all-reduce of the
2P + 3 per-rank partial sums (sum E O, sum O, sum E, sum E^2, n) is enough.
The sums and their combination run in the library (vqnqs_energy_grad_partials,
vqnqs_energy_grad_combine); this module only moves the vector through
torch.distributed (NCCL between GPUs).
"""
from __future__ import annotations


def energy_gradient(model, spins, e_loc, group=None):
    """(grad [P] float32, [mean, var] float64) of the energy over every rank's samples.

    ``model`` provides energy_grad_partials(spins, e_loc) -> float64 [2P + 3] and
    energy_grad_combine(partials) -> (grad, mean_var) (paper_2212_11296_gb300.VQNQS).
    With torch.distributed initialised, the partials are summed over ``group`` (the
    default group when None) by one all-reduce; otherwise the local sums are used."""
    import torch.distributed as dist

    partials = model.energy_grad_partials(spins, e_loc)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(partials, op=dist.ReduceOp.SUM, group=group)
    return model.energy_grad_combine(partials)
