"""Host logic of the multi-GPU form: frames are independent units, so each
rank (one process per GPU) estimates its own share and no collective touches
the data path; ranks only agree on the timed region (barrier) and on the
slowest rank's time (max reduction), from which the whole-job throughput is
computed."""
from __future__ import annotations


def frames_of_rank(n_frames, rank, world):
    """Round-robin share of frame indices 0..n_frames-1 for `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of %d" % (rank, world))
    return list(range(rank, n_frames, world))


def max_over_ranks(value, device=None):
    """The maximum of a float over all ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max, world):
    """Throughput of the job: the units every rank processed over the slowest
    rank's time (weak scaling: each rank processes the same amount)."""
    return world * units_per_rank / seconds_max
