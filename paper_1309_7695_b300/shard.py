"""Sharding of a simulation sweep over ranks, one process per GPU.

The simulations of a sweep are mutually independent (Methods, last
paragraph), so a multi-GPU run needs no exchange on the data path: rank r of
W owns a contiguous range of global simulation indices and writes its own
slice of the outputs.  A simulation's random stream is keyed by its global
index (the ``sim_offset`` of the C ABI), so the union of the shards equals
the unsharded run bit for bit.  The only collectives are the end-of-run
reductions of the timing (maximum over ranks) and of the counters (sum).
"""
from __future__ import annotations


def shard_range(rank: int, world: int, n_total: int) -> tuple[int, int]:
    """[start, stop) of the global indices owned by `rank` when n_total
    simulations are split into `world` contiguous, near-equal parts."""
    if world < 1 or not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad rank/world/n_total")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def weak_offset(rank: int, n_per_rank: int) -> int:
    """Global index of rank's first simulation when every rank simulates its
    own n_per_rank simulations (weak scaling)."""
    return rank * n_per_rank


def reduce_run(seconds: float, counts, device=None):
    """(max over ranks of `seconds`, per-entry sum over ranks of `counts`).

    Uses the default process group when one is initialised (gloo on the CPU,
    NCCL with `device` a CUDA device); otherwise returns the inputs."""
    import torch
    import torch.distributed as dist

    counts = [float(c) for c in counts]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), counts
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    c = torch.tensor(counts, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(v) for v in c.tolist()]
