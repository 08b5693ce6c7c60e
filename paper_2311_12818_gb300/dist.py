"""Multi-process helpers: one process per GPU, chains partitioned across ranks.

Chains are independent, so the walk, contribution and trials need no
collective.  Three things cross ranks:
  - the guide histograms of a training pass (each rank adds its own records;
    the pass's guide is the sum).  Counts are integers, so the sum is exact and
    independent of the reduction order: every rank ends with the same bits.
  - the records of a pass for the vMF guide (and its spatial tree): lobes are
    built from all records, so the ranks' records are gathered in rank order
    and every rank builds the same guide from the same concatenation.
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


def allgather_records(arrays, counts=None, group=None):
    """Concatenation in rank order of every rank's records: `arrays` is a list
    of tensors whose first dimension indexes the records (the same dtypes and
    trailing shapes on every rank), `counts` the number of valid leading
    records per rank (default: all).  Returns the gathered tensors; a stable
    build from them is then identical on every rank."""
    n = int(arrays[0].shape[0]) if counts is None else int(counts)
    mine = torch.tensor([n], dtype=torch.int64, device=arrays[0].device)
    world = dist.get_world_size(group)
    sizes = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(sizes, mine, group=group)
    sizes = [int(x.item()) for x in sizes]
    top = max(sizes)
    out = []
    for a in arrays:
        pad = torch.zeros((top,) + tuple(a.shape[1:]), dtype=a.dtype, device=a.device)
        pad[:n] = a[:n]
        parts = [torch.zeros_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        out.append(torch.cat([p[:sz] for p, sz in zip(parts, sizes)]))
    return out
