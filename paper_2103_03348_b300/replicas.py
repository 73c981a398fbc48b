"""Multi-GPU as independent replicas.

The fused evaluation needs no exchange between GPUs for the benchmark's
purpose: every rank evaluates its own copy of the workload.  The job's
throughput is therefore the units all ranks processed divided by the slowest
rank's time.  These helpers do that reduction over torch.distributed (NCCL on
GPUs, gloo on CPUs in the tests).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> int:
    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def max_over_ranks(value: float, device=None) -> float:
    """The largest value of a per-rank float (the slowest step time)."""
    if world() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: float, ms_local: float, device=None):
    """(job throughput in units/s, slowest rank's ms): weak scaling over replicas."""
    ms = max_over_ranks(ms_local, device)
    return world() * units_per_rank / (ms * 1e-3), ms


def barrier():
    if world() > 1:
        dist.barrier()
