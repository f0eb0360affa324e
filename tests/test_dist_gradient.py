"""The sharded energy gradient's exchange step (paper_2212_11296_gb300.dist) on
CPU with gloo, world size 2 and 3.

Each rank holds its own samples' local energies E_b and per-sample gradients
O_b (random here); a stand-in for the library entry points forms the 2P + 3
partial sums (sum E O, sum O, sum E, sum E^2, n) and combines them as
vqnqs_energy_grad_combine documents.  After the one all-reduce the combined
gradient must equal the single-process formula 2 mean[(E - mean E) O] of the
oracle (oracle.gradient.energy_gradient) on all ranks' samples together, on
every rank, including a rank without samples."""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


class _FakeModel:
    """energy_grad_partials / energy_grad_combine on CPU tensors (float64)."""

    def __init__(self, O):
        self.O = O  # [B_rank, P] float64

    def energy_grad_partials(self, spins, e_loc):
        e = e_loc.double()
        P = self.O.shape[1]
        part = torch.zeros(2 * P + 3, dtype=torch.float64)
        part[:P] = (e[:, None] * self.O).sum(0)
        part[P:2 * P] = self.O.sum(0)
        part[2 * P] = e.sum()
        part[2 * P + 1] = (e * e).sum()
        part[2 * P + 2] = float(len(e))
        return part

    def energy_grad_combine(self, part):
        P = (part.numel() - 3) // 2
        n = part[2 * P + 2]
        mean = part[2 * P] / n
        grad = 2.0 * (part[:P] - mean * part[P:2 * P]) / n
        return grad, torch.stack([mean, part[2 * P + 1] / n - mean * mean])


def _data(n_total, P):
    rng = np.random.default_rng(42)
    return rng.normal(-100.0, 5.0, n_total), rng.normal(size=(n_total, P))


def _worker(rank, world, port, counts, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2212_11296_gb300.dist import energy_gradient
    E, O = _data(sum(counts), 7)
    lo = sum(counts[:rank])
    sl = slice(lo, lo + counts[rank])
    m = _FakeModel(torch.as_tensor(O[sl]))
    grad, mv = energy_gradient(m, None, torch.as_tensor(E[sl]))
    out.put((rank, grad.numpy(), mv.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def _run(counts):
    from oracle import gradient
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = len(counts)
    port = 29600 + (os.getpid() + 7 * world) % 1000
    procs = [ctx.Process(target=_worker, args=(r, world, port, counts, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    E, O = _data(sum(counts), 7)
    want = gradient.energy_gradient(O, E)
    for rank, grad, mv in res:
        np.testing.assert_allclose(grad, want, rtol=1e-9, atol=1e-9)
        assert abs(mv[0] - E.mean()) <= 1e-9 * abs(E.mean())
        assert abs(mv[1] - E.var()) <= 1e-6 * E.var()


def test_two_ranks_one_exchange_equals_single_process():
    _run([5, 8])


def test_three_ranks_one_without_samples():
    _run([4, 0, 6])
