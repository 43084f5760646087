"""Source sharding over replicas (one process per GPU).

The truncated-solver path shards by sources: every replica holds the whole
gauge field and solves a disjoint range of source ids, and the only exchange
is one final sum of the per-set loop accumulators.  These helpers hold that
rule and the timing reduction used by bench.py; they run over any
torch.distributed backend (nccl on GPUs, gloo in the CPU tests).
"""
import torch


def shard(n, rank, world):
    """Contiguous share [first, first + count) of n source ids for `rank`."""
    base, extra = divmod(n, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def sum_over_ranks(array, device="cpu"):
    """Sum of a numpy array over all ranks (identity without a process group)."""
    import numpy as np
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return np.array(array, copy=True)
    t = torch.from_numpy(np.ascontiguousarray(array)).to(device)
    if t.is_complex():
        t = torch.view_as_real(t).contiguous()
        dist.all_reduce(t)
        return torch.view_as_complex(t).cpu().numpy()
    dist.all_reduce(t)
    return t.cpu().numpy()


def max_over_ranks(x, device="cpu"):
    """Largest value of a float over all ranks (the timed region's wall time)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
