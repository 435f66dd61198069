"""Partition of a monostatic RCS sweep over GPUs (one process per GPU).

Monostatic angles are independent problems: each angle has its own ray
screen, trace and Eq. 14 field sum, and the fused geometry is the same input
for all of them.  So ranks share nothing on the data path.  Scaling is weak:
every rank keeps the one-GPU sweep's angle count, and the job's sweep is
`world` times denser in phi.  Rank r takes the r-th interleave (phi shifted
by r / world of the sweep's phi step), so no two ranks compute the same
angle.  The only cross-rank operations are the barrier around the timed
region and the reduction of the ranks' unit counts (sum) and times (max)
into the job's throughput.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def phi_step(phi_deg: np.ndarray) -> float:
    """The sweep's phi spacing (degrees): the smallest positive difference of
    consecutive angles, or 1 degree for a single angle."""
    phi = np.asarray(phi_deg, dtype=np.float64)
    if phi.size < 2:
        return 1.0
    d = np.diff(phi)
    d = d[d > 0]
    return float(d.min()) if d.size else 1.0


def rank_angles(theta_deg, phi_deg, rank: int, world: int) -> Tuple[np.ndarray, np.ndarray]:
    """This rank's (theta, phi) in degrees: the one-GPU sweep with phi
    shifted by rank / world of its step."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError(f"rank {rank} of world {world}")
    th = np.asarray(theta_deg, dtype=np.float64).copy()
    ph = np.asarray(phi_deg, dtype=np.float64) + phi_step(phi_deg) * rank / world
    return th, ph


def job_throughput(units: float, t_ms: float, device=None) -> Tuple[float, float, float]:
    """(units of all ranks, max time over ranks in ms, units per second).

    With torch.distributed initialised and more than one rank, the counts
    are summed and the times reduced by max (the job ends with its slowest
    rank); otherwise the rank's own numbers are returned."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        u = torch.tensor([float(units)], dtype=torch.float64, device=device)
        t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        units, t_ms = float(u.item()), float(t.item())
    return units, t_ms, units / (t_ms / 1e3) if t_ms > 0 else 0.0
