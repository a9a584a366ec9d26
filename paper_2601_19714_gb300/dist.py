"""Multi-GPU layout of the imaging path: channels are independent dirty
images, so ranks take contiguous channel blocks and exchange nothing on the
data path.  The only collectives are the timing barrier and the max over
ranks of a step time (NCCL on GPUs, gloo on the host)."""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def channel_block(total: int, world: int, rank: int):
    """Channels [c0, c1) of rank ``rank``: contiguous blocks whose sizes
    differ by at most one and together cover [0, total) once."""
    if not (0 <= rank < world) or total < 0:
        raise ValueError("rank out of range")
    base, extra = divmod(total, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of ``value`` over all ranks (the value itself when not
    distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
