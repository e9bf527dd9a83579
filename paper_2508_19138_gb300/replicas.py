"""Energy-replica bookkeeping for runs on several GPUs (one process per GPU).

Energies are independent (each energy point is its own selected inversion), so a multi-GPU run
is N replicas: every rank solves its own energies and no data moves between ranks on the
solve path.  The only cross-rank steps are host-side: a barrier around a timed region and the
maximum of the per-rank times.  These helpers hold that logic so it can be exercised with the
gloo backend on CPU."""
from __future__ import annotations

from typing import Tuple


def energy_slice(rank: int, world: int, n_energies: int) -> Tuple[int, int]:
    """Contiguous [begin, end) range of energies owned by `rank` (sizes differ by at most 1)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(n_energies, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def batch_index(rank: int, step: int, n_batches: int) -> int:
    """Which energy batch a rank solves at a given benchmark step (ranks start far apart)."""
    return (rank * 7919 + step) % max(1, n_batches)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
