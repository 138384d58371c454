"""Energy sharding across ranks (one process per GPU).

Energy points are independent (each one is a complete FIND pass), so ranks
take disjoint contiguous blocks of the energy grid and no data moves between
GPUs while they work; the outputs are concatenated on the host afterwards.
The only collectives are host-side: the max of the timed interval and the
final gather, both through whatever torch.distributed backend the caller set
up (NCCL on GPUs, gloo in the CPU tests).
"""

from __future__ import annotations

import numpy as np


def shard_bounds(n_energies: int, rank: int, world: int):
    """[lo, hi) of this rank's contiguous block; blocks differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_energies, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def step_energies(energies: np.ndarray, step: int, rank: int, world: int, batch: int) -> np.ndarray:
    """Energies of one benchmark step on one rank: consecutive batches, rank
    after rank, wrapping around the grid."""
    idx = ((step * world + rank) * batch + np.arange(batch)) % len(energies)
    return np.ascontiguousarray(energies[idx])


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the timed interval of a step)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_outputs(local: np.ndarray, n_energies: int):
    """Concatenate every rank's block (rank order) on every rank, on the host."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, np.asarray(local))
    out = np.concatenate(parts, axis=0)
    if out.shape[0] != n_energies:
        raise RuntimeError("gathered energy count does not match the grid")
    return out


def solve_sharded(solve, energies: np.ndarray, rank: int, world: int):
    """Run `solve(local_energies) -> array (n_local, ...)` on this rank's block
    and return the whole grid's outputs, gathered on the host."""
    lo, hi = shard_bounds(len(energies), rank, world)
    local = np.asarray(solve(np.ascontiguousarray(energies[lo:hi])))
    return gather_outputs(local, len(energies))
