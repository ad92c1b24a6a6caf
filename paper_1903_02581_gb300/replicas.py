"""Replicas on several GPUs: one process per GPU, no data-path collective.

A single simulation does not shard without an all-to-all transpose of the
state in every step, so N processes propagate N independent workloads (weak
scaling): the full-scale grid with the packet widths sigma = 2, 1, 4 (cycled
over the ranks), or disjoint blocks of the batched sweep.  The only
collectives are the barriers around a timed region and one max-reduction of
its elapsed time; the whole-job rate divides all ranks' updates by the
slowest rank's time.
"""

from __future__ import annotations

from . import workloads as W

FULLSCALE_SIGMAS = (2.0, 1.0, 4.0)


def rank_workload(kind: str, rank: int) -> tuple[dict, str]:
    """The workload rank ``rank`` propagates, and its name."""
    if rank < 0:
        raise ValueError("rank must be >= 0")
    if kind == "batched":
        return W.batched(shard=rank), "batched-32x128x32"
    if kind == "fullscale":
        return W.fullscale(sigma=FULLSCALE_SIGMAS[rank % len(FULLSCALE_SIGMAS)]), "fullscale-256x64"
    raise ValueError(f"unknown workload {kind!r}")


def slowest(value: float, device=None) -> float:
    """The maximum of ``value`` over the ranks of the default process group
    (``value`` itself without one); ``device`` holds the reduction buffer
    (a CUDA device for NCCL, None for the CPU with gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, sims_per_rank: int, points_per_sim: int, steps: int, seconds: float) -> float:
    """Whole-job grid-point updates per second: every rank's updates over the
    slowest rank's time."""
    if seconds <= 0:
        raise ValueError("seconds must be > 0")
    return world * sims_per_rank * points_per_sim * steps / seconds
