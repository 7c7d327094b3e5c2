"""Walker sharding across GPUs, one process per GPU.

Walkers (with their tethered paths) are independent within a step, and every
random draw is addressed by the walker's global index (the library's
``walker_offset``), so splitting one population into contiguous blocks of
walkers reproduces the single-GPU run exactly.  The only exchange is the
mixed-estimator sums {sum W Re E, sum W, sum W |sum S|/P} of each measured step,
three doubles, summed over ranks; for the estimate from extra measurement paths
(afqmc_energy_paths), the complex sums {sum W R E', sum W R}.  With population
control on (pop_period > 0) every GPU combs its own walkers, with no walker
exchange, so a sharded run is a different (equally valid) population from the
single-GPU one from the first comb on.
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


def combine_paths(weight, e_walker, ratio, group=None) -> float:
    """Global estimate from extra measurement paths: each rank passes its
    walkers' weights W_w and the E'_w and R_w that afqmc_energy_paths returned
    (R_w = 0 for walkers that do not count); returns
    Re(sum W R E' / sum W R) over all ranks."""
    import numpy as np
    import torch
    import torch.distributed as dist
    wr = np.asarray(weight, dtype=np.float64) * np.asarray(ratio, dtype=np.complex128)
    num = np.sum(wr * np.asarray(e_walker, dtype=np.complex128))
    den = np.sum(wr)
    dev = "cpu"
    if dist.is_initialized() and dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([num.real, num.imag, den.real, den.imag], dtype=torch.float64, device=dev)
    if dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    nr, ni, dr, di = t.tolist()
    q = complex(nr, ni) / complex(dr, di) if (dr, di) != (0.0, 0.0) else 0.0
    return float(np.real(q))


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
