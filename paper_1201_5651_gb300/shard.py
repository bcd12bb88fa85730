"""Substeps split over processes: sources for the traces, z-slabs of cells for
the per-cell passes (Mackey 2012, Sect. 5: the domain is decomposed and each
source's rays are traced outward across it; sources and octants are traced
independently).

One process per GPU.  Process r traces the sources it owns (round robin) and
integrates the cells of its z-slab; every process keeps the whole state and
all columns, exchanged between the phases of a substep:

    trace x (own sources)  -> broadcast each source's columns from its owner
    Eq. 4 on own cells     -> minimum over processes (all-reduce)
    A3: half step on own cells -> broadcast each slab of x_half from its owner
        trace x_half (own sources) -> broadcast the second columns
        full step on own cells
    A2: the step on own cells
    broadcast each slab of x from its owner

The phases run through the C ABI (oots_set_partition, oots_run_phase,
oots_array_device; ContextBackend); the exchanges through a Comm: TorchComm
(torch.distributed: NCCL between GPUs, gloo on host memory) or ThreadComm
(several partitions driven by threads of one process).  Any object with the
backend's methods can stand in for a context, which is how the host logic is
tested without a GPU.
"""
from __future__ import annotations

import threading
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import oots

KIND_X, KIND_XH, KIND_N1, KIND_N2 = 0, 1, 2, 3


def source_masks(nsrc: int, size: int) -> List[int]:
    """Sources per process, round robin: bit s of mask r is set when process r traces source s."""
    masks = [0] * size
    for s in range(nsrc):
        masks[s % size] |= 1 << s
    return masks


def source_owner(nsrc: int, size: int) -> List[int]:
    return [s % size for s in range(nsrc)]


def z_slabs(nz: int, size: int) -> List[Tuple[int, int]]:
    """Contiguous z-ranges, as even as the planes allow, one per process."""
    base, extra = divmod(nz, size)
    out, z = [], 0
    for r in range(size):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


class TorchComm:
    """Exchanges between processes through torch.distributed (the default group)."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.torch = torch
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()
        self.device = device if device is not None else "cpu"

    def broadcast(self, tensor, src: int) -> None:
        self.dist.broadcast(tensor, src=src)

    def allreduce_min(self, v: float) -> float:
        t = self.torch.tensor([v], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN)
        return float(t.item())


class ThreadGroup:
    """Shared state of the ThreadComms of one process."""

    def __init__(self, size: int):
        self.size = size
        self.barrier = threading.Barrier(size)
        self.slot: Dict[int, object] = {}
        self.vals: List[float] = [0.0] * size


class ThreadComm:
    """Exchanges between partitions driven by the threads of one process.
    Tensors are torch tensors (any device); a broadcast copies the source's
    tensor into every other partition's."""

    def __init__(self, group: ThreadGroup, rank: int):
        self.g = group
        self.rank = rank
        self.size = group.size

    def broadcast(self, tensor, src: int) -> None:
        g = self.g
        if self.rank == src:
            g.slot[src] = tensor
        g.barrier.wait()
        if self.rank != src:
            tensor.copy_(g.slot[src])
            if tensor.is_cuda:
                import torch
                torch.cuda.current_stream(tensor.device).synchronize()
        g.barrier.wait()

    def allreduce_min(self, v: float) -> float:
        g = self.g
        g.vals[self.rank] = v
        g.barrier.wait()
        m = min(g.vals)
        g.barrier.wait()
        return m


class _CudaArray:
    """__cuda_array_interface__ over a context's device array (no copy)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2,
                                         "strides": None}


class ContextBackend:
    """One process's share of a partitioned run on its GPU, through the C ABI."""

    def __init__(self, ctx: "oots.Context", src_mask: int, z0: int, z1: int):
        self.ctx = ctx
        ctx.set_partition(src_mask, z0, z1)
        nz, ny, nx = ctx.shape
        self.ncell = nx * ny * nz
        self.plane = nx * ny

    def trace(self, which: int) -> None:
        self.ctx.run_phase(oots.OOTS_PH_TRACE1 if which == 0 else oots.OOTS_PH_TRACE2)

    def dt_local(self) -> float:
        return self.ctx.run_phase(oots.OOTS_PH_DT)

    def step1(self, dt: float) -> None:
        self.ctx.run_phase(oots.OOTS_PH_STEP1, dt)

    def full(self) -> None:
        self.ctx.run_phase(oots.OOTS_PH_FULL)

    def time(self) -> float:
        return self.ctx.get_time()[0]

    def array(self, kind: int, source: int = 0):
        import torch
        ptr, nbytes = self.ctx.array_device(kind, source)
        typestr = "<f8" if self.ctx.precision == oots.OOTS_FP64 else "<f4"
        return torch.as_tensor(_CudaArray(ptr, nbytes // (8 if typestr == "<f8" else 4), typestr), device="cuda")

    def exchanged(self) -> None:
        # the exchanges ran on torch's stream; the next phase runs on the context's
        import torch
        torch.cuda.synchronize()


class ShardedRun:
    """Drives the substeps of one process of a partitioned run (see the module text)."""

    def __init__(self, backend, comm, nsrc: int, nz: int, scheme: int = oots.OOTS_A3):
        self.b = backend
        self.comm = comm
        self.nsrc = nsrc
        self.scheme = scheme
        self.owner = source_owner(nsrc, comm.size)
        self.slabs = z_slabs(nz, comm.size)
        self.plane = backend.plane

    def _share_columns(self, kind: int) -> None:
        for s in range(self.nsrc):
            self.comm.broadcast(self.b.array(kind, s), self.owner[s])

    def _share_state(self, kind: int) -> None:
        a = self.b.array(kind)
        for r, (z0, z1) in enumerate(self.slabs):
            if z1 > z0:
                self.comm.broadcast(a[z0 * self.plane:z1 * self.plane], r)

    def substep(self, t_end: float) -> float:
        """One substep toward t_end on every process; returns the step taken (0: at t_end)."""
        t = self.b.time()
        if not t < t_end:
            return 0.0
        self.b.trace(0)
        self._share_columns(KIND_N1)
        self.b.exchanged()
        dt = self.comm.allreduce_min(self.b.dt_local())
        rem = t_end - t
        if dt >= rem * (1.0 - 1e-12):
            dt = rem
        self.b.step1(dt)
        if self.scheme == oots.OOTS_A3:
            self._share_state(KIND_XH)
            self.b.exchanged()
            self.b.trace(1)
            self._share_columns(KIND_N2)
            self.b.exchanged()
            self.b.full()
        self._share_state(KIND_X)
        self.b.exchanged()
        return dt

    def advance(self, t_end: float, max_steps: int = 10 ** 9) -> int:
        n = 0
        while n < max_steps and self.substep(t_end) > 0.0:
            n += 1
        return n


def run_threads(contexts: Sequence["oots.Context"], nsrc: int, t_end: float, scheme: int = oots.OOTS_A3,
                max_steps: int = 10 ** 9) -> List[int]:
    """Drive len(contexts) partitions of one problem from threads of this process
    (one context per partition, e.g. one per GPU), each with its own share."""
    size = len(contexts)
    nz = contexts[0].shape[0]
    masks = source_masks(nsrc, size)
    slabs = z_slabs(nz, size)
    group = ThreadGroup(size)
    out = [0] * size
    errs: List[BaseException] = []

    def work(r):
        try:
            b = ContextBackend(contexts[r], masks[r], *slabs[r])
            out[r] = ShardedRun(b, ThreadComm(group, r), nsrc, nz, scheme).advance(t_end, max_steps)
        except BaseException as e:          # noqa: BLE001 -- reported below, the barrier released
            errs.append(e)
            group.barrier.abort()

    th = [threading.Thread(target=work, args=(r,)) for r in range(size)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return out
