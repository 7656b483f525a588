"""Many GPUs: the cast shards by rays.

Rays are independent and the tally is a sum of per-ray scores (Eq. 4), so N
ranks (one process per GPU) each cast their own share of the rays into their
own tally; the only exchange is one sum of the tallies when the result is
read (the paper reads the tally once, at the end of the run, Sec. 3).  There
is no collective inside the cast.

shard(): the contiguous share of a batch that rank r of N casts.
allreduce_tally(): sums the float64 tallies of every rank in place
(torch.distributed: NCCL for device tensors, gloo for host tensors).
"""
from __future__ import annotations


def shard(n: int, rank: int, world: int) -> slice:
    """Rays [n*rank//world, n*(rank+1)//world) of an n-ray batch."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return slice(n * rank // world, n * (rank + 1) // world)


def allreduce_tally(tally, group=None):
    """Sums a float64 tally tensor over all ranks of the process group."""
    import torch
    import torch.distributed as dist
    if tally.dtype != torch.float64:
        raise TypeError("tallies are float64")
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    return tally


def device_tally(vrc, ctx):
    """The context's device tally as a torch float64 CUDA tensor (no copy)."""
    import torch
    ptr = vrc.vrc_tally_device_ptr(ctx)
    # a view of the library-owned buffer; valid until the context is destroyed
    return torch.as_tensor(_CudaArray(ptr, ctx.tally_size), device="cuda")


class _CudaArray:
    """__cuda_array_interface__ view of a libvrc float64 device buffer."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None}
