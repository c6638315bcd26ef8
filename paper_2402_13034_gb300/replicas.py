"""Replicas over several GPUs (one process per GPU): the field path shards by receivers with no
exchange step, so every rank traces and evaluates its own receiver batch and only the timing is
combined. Host logic only; works with any torch.distributed backend (NCCL on GPUs, gloo on CPU)."""
from __future__ import annotations

import numpy as np


def rank_receivers(rx_xyz: np.ndarray, rank: int, shift_m: float = 1e-3) -> np.ndarray:
    """Rank r's receiver batch: the workload's grid moved by r * shift_m along x (weak scaling: every
    rank has a batch of the same size and structure, distinct from the others')."""
    out = np.array(rx_xyz, dtype=np.float32, copy=True)
    if rank:
        out[:, 0] += np.float32(shift_m * rank)
    return out


def combine_over_ranks(elapsed_ms: float, units: float, device="cpu") -> tuple[float, float]:
    """Whole-job timing of a weak-scaling run: the slowest rank's elapsed time and the units of all
    ranks. Without an initialised process group it returns its arguments."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_ms), float(units)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
