"""Multi-GPU form of the benchmark: independent replicas, one per rank.

The IBM step of one case does not need a collective; with several GPUs each
rank advances its own case (the Mach 0.3 heated sphere with a hot or a cold
wall, alternating over ranks) and only the timings are combined: the job
time is the maximum over ranks, the work the sum (weak scaling).  The Mach 2
variants are not used here: started impulsively from a uniform stream they
reach a non-positive pressure within 100 steps at 256^3.
"""
from __future__ import annotations

from . import cases


def case_for_rank(rank: int, world: int, n: int = 256) -> cases.Case:
    variants = [v for v in cases.sphere_variants(n) if v.grid.Mach < 1.0]
    return variants[0] if world == 1 else variants[rank % len(variants)]


def reduce_timings(dist, device, ms: float, e2e_ms: float, cells: float, markers: float):
    """Max of the times and sum of the work over ranks (no-op for one rank).
    Returns (ms_max, e2e_ms_max, cells_sum, markers_sum)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, e2e_ms, cells, markers
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    w = torch.tensor([cells, markers], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(w[0]), float(w[1])
