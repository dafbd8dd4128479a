"""One plasma split over several processes by markers (one GPU each).

The markers of the scheme are independent of each other given the fields, and
the fields depend on them only through sums over markers: the charge of the
discrete Poisson equation, each subsystem-I sweep's current deposit, each
subsystem-II sweep's susceptibility deposit and the spin source (Sec. 4.2),
and the kinetic and Zeeman energies.  So a plasma too large for one GPU is split
by markers: every process holds a contiguous share of them and the same fields,
and after each such sum an all-reduce over the processes makes the sums global;
the fixed-point test takes the largest marker increment over all processes the
same way.  Every process then solves the same grid equations and takes the same
decisions.  The library (pic_init_split in include/pic.h) calls back into this
module for each reduction; here the reduction is torch.distributed's all_reduce
(NCCL between GPUs, gloo on CPU tensors), issued on the handle's stream.

This module holds no arithmetic of the method.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import pic

PIC_REDUCE_SUM, PIC_REDUCE_MAX = 0, 1

REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_void_p)


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous marker range [lo, hi) of process `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    return n * rank // world, n * (rank + 1) // world


class TorchComm:
    """Sums and maxima over the processes of a torch.distributed group, on host
    (numpy) values; the CPU reference of the split uses it."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group

    def sum(self, a: np.ndarray) -> np.ndarray:
        import torch
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).copy())
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.numpy()

    def max(self, v: float) -> float:
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())


class _DeviceArray:
    """A device array of n doubles at a raw address, as torch sees it."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class TorchDeviceReducer:
    """The library's reduction callback over torch.distributed on CUDA tensors:
    an in-place all_reduce of the buffer, issued on the handle's stream."""

    def __init__(self, group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.error = None
        self.cfunc = REDUCE_FN(self._call)

    def _call(self, ctx, op, ptr, n, stream):
        try:
            torch, dist = self.torch, self.dist
            t = torch.as_tensor(_DeviceArray(ptr, n), device="cuda")
            s = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(s):
                dist.all_reduce(t, op=dist.ReduceOp.SUM if op == PIC_REDUCE_SUM else dist.ReduceOp.MAX,
                                group=self.group)
            return 0
        except Exception as e:          # reported by the library as a failed reduction
            self.error = e
            return 1


def init_split(cfg: "pic.Config", x, p, ay, az, ey=None, ez=None, stream=None, spin=None,
               reducer=None) -> "pic.Pic":
    """A handle on this process's share of the markers (cfg.np = the local count,
    cfg.weight = L / the global count); `reducer` provides `cfunc` (the C
    callback, kept alive by the returned object)."""
    return pic.Pic(cfg, x, p, ay, az, ey, ez, stream=stream, spin=spin, reducer=reducer)
