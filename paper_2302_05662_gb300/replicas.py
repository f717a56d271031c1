"""Host logic of running the benchmark step as independent replicas, one per
GPU (the single product would shard by row blocks with an all-gather of x;
the benchmark instead runs whole independent products per rank, so there is
no data-path collective).  The only communication is the timing: a barrier
before and after the timed region and the maximum of the ranks' elapsed
times, from which the whole-job throughput is formed."""
from __future__ import annotations


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, steps: int, world: int, elapsed_ms_max: float) -> float:
    """Units per second of the whole job: every rank processes
    units_per_rank per step; the job takes the slowest rank's time."""
    return units_per_rank * steps * world / (elapsed_ms_max * 1e-3)
