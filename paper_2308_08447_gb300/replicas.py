"""Replica bookkeeping for multi-GPU runs of independent meshes.

Meshes never exchange data, so N ranks run N independent replicas (one process per GPU, no
collective on the data path). The only cross-rank steps are the timing ones: a barrier around
the timed region, the slowest rank's time (the job's time), and the sum of the work done.
These helpers take an initialised torch.distributed process group (NCCL on GPUs, gloo on CPU),
or none for a single process.
"""


def _dist():
    import torch.distributed as dist
    return dist if (dist.is_available() and dist.is_initialized()) else None


def barrier():
    d = _dist()
    if d is not None:
        d.barrier()


def _reduce(value, op_name, device):
    import torch
    d = _dist()
    if d is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=getattr(d.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(value, device="cpu"):
    """The largest value over all ranks (every rank gets it)."""
    return _reduce(value, "MAX", device)


def sum_over_ranks(value, device="cpu"):
    """The sum over all ranks (every rank gets it)."""
    return _reduce(value, "SUM", device)


def job_throughput(units_per_rank, seconds_per_rank, device="cpu"):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    total = sum_over_ranks(units_per_rank, device)
    t = max_over_ranks(seconds_per_rank, device)
    return total / t, t, total
