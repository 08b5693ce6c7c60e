"""Multi-process helpers: one process per GPU, chains partitioned across ranks.

Chains are independent, so the walk, contribution and trials need no
collective.  Two things cross ranks:
  - the guide histograms of a training pass (each rank adds its own records;
    the pass's guide is the sum).  Counts are integers, so the sum is exact and
    independent of the reduction order: every rank ends with the same bits.
  - the job's throughput: units processed on all ranks over the slowest rank's
    time.
"""
import torch
import torch.distributed as dist

from . import mpg


def sum_histograms(counts: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum over ranks of guide counts (int64 tensors holding the uint64
    counters: two's-complement addition wraps exactly like uint64)."""
    if counts.dtype != torch.int64:
        raise TypeError("guide counts are int64 (uint64 bit patterns)")
    dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts


def allreduce_guide(ctx, guide, group=None, stream=None):
    """Sums the ranks' guide counts, then rebuilds the prefix sums the sampler
    uses (mpg_guide_update with no records)."""
    sum_histograms(guide.counts, group)
    mpg.mpg_guide_update(ctx, guide, None, None, None, R=0, stream=stream)


def job_throughput(t_ms: float, units: float, device="cpu", group=None):
    """(slowest rank's time in ms, units summed over ranks)."""
    if not dist.is_available() or not dist.is_initialized():
        return t_ms, units
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())
