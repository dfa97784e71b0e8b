"""Work partition over ranks (one process per GPU) and assembly of Omega.

Every (partial wave, energy) pair is independent (Section "Overview": the
energy loop is the parallel one; Section "Computational details": v1.1 gives
each processor all energies of every partial wave, never consecutive
energies of one partial wave, and sums the partial collision strengths over
processors with a reduce). Two assignments are provided:

  energy_shard   rank r takes energies r, r+N, ... of the grid for every
                 partial wave. Omega rows of different ranks are disjoint,
                 so the data path needs no collective; gather_omega only
                 assembles the output (used by bench.py under torchrun).
  twisted_shard  the paper's v1.1 assignment: for partial wave p, rank r
                 takes energies m with (m + p) mod N == r, so a rank's slow
                 (half-open) energies differ from one partial wave to the
                 next. Each energy's Omega is then split over ranks and
                 reduce_omega sums it (the paper's MPI_REDUCE).

The collectives use torch.distributed (NCCL on GPUs, gloo on CPU).
"""
import numpy as np


def energy_shard(n_E, rank, world):
    """Indices of the energies of `rank` (interleaved)."""
    return np.arange(rank, n_E, world, dtype=np.int64)


def twisted_shard(n_E, pw, rank, world):
    """Indices of the energies of partial wave `pw` handled by `rank`."""
    return np.arange((rank - pw) % world, n_E, world, dtype=np.int64)


def pw_order(n_pw, rank, world):
    """Order in which `rank` visits the partial waves: each rank starts at a
    different one (the paper staggers the start so ranks do not read the same
    partial wave at the same time)."""
    start = (rank * n_pw) // max(world, 1)
    return [(start + k) % n_pw for k in range(n_pw)]


def gather_omega(local_rows, n_E, rank, world, group=None):
    """Assemble the full [n_E][n_tri] Omega on every rank from the rows each
    rank computed for its energy_shard (torch.distributed all_gather)."""
    import torch
    import torch.distributed as dist

    local = torch.as_tensor(np.ascontiguousarray(local_rows))
    n_tri = local.shape[1]
    per = (n_E + world - 1) // world
    pad = torch.zeros((per, n_tri), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = np.zeros((n_E, n_tri))
    for r in range(world):
        idx = energy_shard(n_E, r, world)
        out[idx] = parts[r][: idx.size].cpu().numpy()
    return out


def reduce_omega(omega, group=None):
    """Sum a full-grid partial Omega over ranks (in place on a torch tensor,
    or returns a new numpy array)."""
    import torch
    import torch.distributed as dist

    t = torch.as_tensor(np.ascontiguousarray(omega)) if not hasattr(omega, "data_ptr") else omega
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t if hasattr(omega, "data_ptr") else t.cpu().numpy()
