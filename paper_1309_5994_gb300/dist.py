"""Multi-process plumbing: one process per GPU, block columns sharded across ranks.

Block columns (source sites) are independent right-hand sides of the Dyson
equation (Sec. IV.D: every unit vector is solved on its own), so ranks share
nothing while they sweep.  The lattice solve needs only host-side bookkeeping:
a barrier and a max-reduction around timed regions, and one final all-gather
that merges per-site observables.  The self-consistency loop of Sec. IV.C has
one real exchange per iteration: every site's self-energy needs the local Green's
functions of its neighbours, which other ranks solved (sum_rows_).
"""
from __future__ import annotations

import os
from typing import List

import numpy as np


def env_ranks():
    """(rank, world_size, local_rank) from the torchrun environment (defaults 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str):
    """Initialise torch.distributed when WORLD_SIZE > 1; returns (rank, world, local)."""
    rank, world, local = env_ranks()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
    return rank, world, local


def step_sources(n_sites: int, batch: int, rank: int, world: int, step: int) -> List[int]:
    """Source sites of one step on one rank: consecutive, disjoint across ranks and
    steps until all n_sites are covered, then wrapping around."""
    base = (step * world + rank) * batch
    return [(base + q) % n_sites for q in range(batch)]


def shard_sites(n_sites: int, rank: int, world: int) -> List[int]:
    """A contiguous, balanced partition of all sites over the ranks."""
    per, extra = divmod(n_sites, world)
    start = rank * per + min(rank, extra)
    return list(range(start, start + per + (1 if rank < extra else 0)))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a host float over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device_index=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device_index is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device_index])
        else:
            dist.barrier()


def merge_observables(parts: List[np.ndarray]) -> np.ndarray:
    """Merge per-rank [.., Nr, Nt] observable arrays whose unsolved sites hold NaN.

    Every site must be solved by exactly one rank (or by several with identical
    values); a site solved nowhere stays NaN."""
    out = np.full_like(parts[0], np.nan)
    for p in parts:
        have = ~np.isnan(p)
        clash = have & ~np.isnan(out) & (out != p)
        if np.any(clash):
            raise ValueError("ranks disagree on a site's observables")
        out[have] = p[have]
    return out


def all_gather_observables(local: np.ndarray, device=None) -> np.ndarray:
    """All-gather a rank's observable array and merge (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local
    t = torch.from_numpy(np.ascontiguousarray(local)).to(device if device is not None else "cpu")
    bufs = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(bufs, t)
    return merge_observables([b.cpu().numpy() for b in bufs])


def sum_rows_(t):
    """In place, sum a tensor over the ranks (each rank holds its own rows, zeros elsewhere,
    so the sum is the merge); a complex tensor travels as its real view.  Identity when not
    distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return t
    dist.all_reduce(torch.view_as_real(t) if t.is_complex() else t, op=dist.ReduceOp.SUM)
    return t
