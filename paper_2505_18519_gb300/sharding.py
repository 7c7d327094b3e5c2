"""Walker sharding across GPUs, one process per GPU.

Walkers (with their tethered paths) are independent within a step, and every
random draw is addressed by the walker's global index (the library's
``walker_offset``), so splitting one population into contiguous blocks of
walkers reproduces the single-GPU run exactly.  The only exchange is the
mixed-estimator sums {sum W Re E, sum W, sum W |sum S|/P} of each measured step,
three doubles, summed over ranks.
"""

from __future__ import annotations


def shard(total_walkers: int, world: int, rank: int):
    """(walker_offset, n_walkers) of ``rank``'s contiguous block of walkers."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(total_walkers, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def combine_mixed(sums, group=None):
    """Sum per-rank mixed-estimator sums (a length-3 sequence) over ranks and
    return (E_mix, sum_w, mean_sign).  Works for any torch.distributed backend;
    the tensor lives on CPU for gloo and on the current CUDA device for NCCL."""
    import torch
    import torch.distributed as dist
    dev = "cpu"
    if dist.is_initialized() and dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([float(v) for v in sums], dtype=torch.float64, device=dev)
    if dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    num, den, sgn = t.tolist()
    return (num / den if den > 0 else 0.0), den, (sgn / den if den > 0 else 0.0)


def max_over_ranks(value: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return float(value)
    dev = "cpu"
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
