"""Multi-GPU replicas: walkers are independent Markov chains (Sec. 2.2), so ranks run
disjoint walker sets and nothing is exchanged on the data path.  This module holds the
host-side bookkeeping: which seeds a rank owns, and the end-of-run reduction of counts
(summed) and elapsed times (maximum over ranks) through torch.distributed."""
from __future__ import annotations


def walker_seeds(rank: int, walkers_per_rank: int, base: int = 1) -> list[int]:
    """Seeds of rank `rank`: walker w of rank r is global walker r * walkers_per_rank + w,
    seeded base + global index (so rank 0 reproduces the single-GPU seeds)."""
    if rank < 0 or walkers_per_rank <= 0:
        raise ValueError("rank >= 0 and walkers_per_rank > 0 required")
    return [base + rank * walkers_per_rank + w for w in range(walkers_per_rank)]


def reduce_run(count: float, elapsed: float, device=None):
    """(sum of counts over ranks, max of elapsed over ranks); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(count), float(elapsed)
    dev = device if device is not None else ("cuda" if dist.get_backend() == "nccl" else "cpu")
    c = torch.tensor([float(count)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=dev)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(c.item()), float(t.item())


def throughput(count: float, elapsed_s: float) -> float:
    """Whole-job rate: all ranks' work over the slowest rank's time."""
    return count / elapsed_s if elapsed_s > 0 else float("inf")
