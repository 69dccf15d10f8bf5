"""Frequency sharding over GPUs (Sec. IV-D: sources spread over workers,
partial Jacobian products aggregated).

Each rank (one process per GPU) creates its libfwi context with a subset of
the frequencies -- every transmit of each -- and the matching rows of the
observed data.  The sums over frequencies in the misfit, the gradient and
each Gauss-Newton CG iteration's J^H J d are completed by a reducer that
the library calls (fwi_set_reducer); the reducers here sum over the ranks of
a torch.distributed process group:

* ``collective_reducer``: all_reduce of the device buffer itself, ordered on
  the context's CUDA stream (NCCL);
* ``host_staged_reducer``: copy to host on the context's stream, all_reduce
  there (any backend, e.g. gloo), copy back on the stream.

These are argument marshalling around torch.distributed: the library's
kernels do the arithmetic, the process group the communication."""
import ctypes

import numpy as np


def frequency_shard(n_freq, world, rank):
    """Frequencies of ``rank``: l = rank, rank + world, ... (round robin, so
    that low and high frequencies, whose solves take fewer and more Krylov
    iterations, are spread over the ranks)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(range(rank, n_freq, world))


class _CudaArray:
    """A device buffer of float64 values exposed through
    __cuda_array_interface__ (zero copy)."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def device_array(ptr, count):
    """torch float64 CUDA tensor aliasing ``count`` doubles at ``ptr``."""
    import torch
    return torch.as_tensor(_CudaArray(ptr, count), device="cuda")


def host_array(ptr, count):
    """torch float64 CPU tensor aliasing ``count`` doubles at host address
    ``ptr``."""
    import torch
    buf = (ctypes.c_double * int(count)).from_address(int(ptr))
    return torch.from_numpy(np.ctypeslib.as_array(buf))


def collective_reducer(group=None, wrap=device_array):
    """Reducer: torch.distributed all_reduce (sum) of the buffer in place,
    issued with the context's stream current (NCCL orders the collective
    after the work on that stream and the stream's later work after it)."""
    import torch
    import torch.distributed as dist

    def reduce(ptr, count, stream):
        t = wrap(ptr, count)
        if t.is_cuda:
            with torch.cuda.stream(torch.cuda.ExternalStream(stream, device=t.device)):
                dist.all_reduce(t, group=group)
        else:
            dist.all_reduce(t, group=group)
    return reduce


def host_staged_reducer(group=None, wrap=device_array):
    """Reducer through host memory: blocking copy of the buffer to the host
    on the context's stream, all_reduce (sum) on the host copy, copy back on
    the stream.  Works with any backend (gloo)."""
    import torch
    import torch.distributed as dist

    def reduce(ptr, count, stream):
        t = wrap(ptr, count)
        if not t.is_cuda:
            dist.all_reduce(t, group=group)
            return
        s = torch.cuda.ExternalStream(stream, device=t.device)
        with torch.cuda.stream(s):
            h = t.to("cpu")
            dist.all_reduce(h, group=group)
            t.copy_(h)
    return reduce
