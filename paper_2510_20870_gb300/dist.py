"""Multi-GPU plumbing: the cross-section path needs no exchange between GPUs.

(P,T) points are independent, and so are wavenumber windows given the lines within the cutoff
of them, so N GPUs run N independent shares of a workload (or N replicas of it) and the only
communication is host-side: a barrier, the maximum of the ranks' step times, and gathering
disjoint output slices. No collective touches the data path. These helpers hold that host
logic so that it can be tested on CPU ranks (gloo) as well as used by bench.py (NCCL).
"""
import torch


def split_range(n, world, rank):
    """Contiguous share [a, b) of range(n) for this rank (sizes differ by at most one)."""
    q, r = divmod(n, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def point_shard(points, world, rank):
    """The (P,T) points this rank computes (contiguous block)."""
    a, b = split_range(len(points), world, rank)
    return points[a:b], a


def span_shard(n_grid, span, world, rank):
    """A wavenumber window [first, first + n) of whole spans for this rank."""
    n_spans = (n_grid + span - 1) // span
    a, b = split_range(n_spans, world, rank)
    first = a * span
    return first, max(0, min(n_grid, b * span) - first)


def max_over_ranks(value, device=None):
    """Max of a float over all ranks (time of the slowest rank); identity without a group."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_slices(local, total_len, first, device=None):
    """Concatenate disjoint 1-D output slices of all ranks into the full array on every rank
    (host-side gather of finished results, not part of the compute path)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local
    full = torch.zeros(total_len, dtype=local.dtype, device=device)
    full[first:first + local.numel()] = local.to(device)
    dist.all_reduce(full, op=dist.ReduceOp.SUM)   # slices are disjoint: the sum is a gather
    return full
