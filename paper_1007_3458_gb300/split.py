"""One system's hybrid step split over several GPUs (one process per GPU).

Every rank holds the whole state of the system. Rank r of W owns a contiguous
block of bodies (``split_rows``): it computes the O(N^2) kick of its rows
against every row (Sec. 2, Eq. 4) with the crude encounter search of those
rows (Sec. 2.4), their Kepler drift (Appendix), the rigorous test of their
candidate pairs, and the Hermite sub-integration (Sec. 2.2-2.3) of the
encounter sets whose lowest row it owns. What every rank needs of the others'
work is exchanged between the phases of the step (``SplitRun.step``):

  after the first kick   v, |a| and the Hill radii of each rank's rows
  after the Kepler drift q1, v1 of each rank's rows
  after the rigorous test every rank's encounter pairs (sets are then built
                         from all of them on every rank)
  after the Hermite      q1, v1 and the block-step counts of the members of
                         each rank's sets
  after the second kick  v and |a| of each rank's rows

The momentum sum and the drifts (Sec. 2, Eq. 2), the kick operand packs and
the encounter sets are computed on every rank from identical data in a fixed
order, so they agree to the bit without a collective.

A rank's compute is an *engine* (``GpuEngine``: one libqym context; the phases
are the library's qym_split_phase); the exchanges go through a *comm* with an
all-gather (``TorchComm``: torch.distributed, NCCL between GPUs). This module
only moves data between ranks: all arithmetic of the step runs in the engine.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import (QYM_PHASE_CLOSE, QYM_PHASE_HERMITE, QYM_PHASE_KEPLER, QYM_PHASE_KICK1,
               QYM_PHASE_KICK2, QYM_PHASE_OPEN, QYM_PHASE_REFINE, QYM_PHASE_SEARCH)


def split_rows(rows: int, rank: int, world: int):
    """Rows [lo, hi) owned by rank of world: the bodies 1 .. rows-1 in
    contiguous blocks of ceil((rows-1) / world), the last one shorter (the
    same blocks as the library's qym_split_rows)."""
    nb = rows - 1
    blk = (nb + world - 1) // world
    lo = min(1 + rank * blk, rows)
    hi = min(lo + blk, rows)
    return lo, hi


class TorchComm:
    """All-gathers over torch.distributed's default process group: NCCL for
    CUDA tensors between GPUs, gloo for CPU tensors."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()

    def allgather(self, t):
        """t: a tensor of the same shape on every rank -> list of world tensors."""
        import torch
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t.contiguous())
        return out


class SplitRun:
    """Drives one rank's engine through the phases of the split step and
    performs the exchanges between them."""

    ROW_ARRAYS_KICK1 = ("v", "amag", "rH")
    ROW_ARRAYS_KEPLER = ("q1", "v1")
    ROW_ARRAYS_KICK2 = ("v", "amag")

    def __init__(self, engine, comm):
        self.e = engine
        self.comm = comm
        self.rank, self.world = comm.rank, comm.world
        self.rows = engine.rows
        self.blocks = [split_rows(self.rows, r, self.world) for r in range(self.world)]
        self.blk = max(1, max(hi - lo for lo, hi in self.blocks))
        if engine.own != self.blocks[self.rank]:
            raise ValueError(f"engine owns rows {engine.own}, expected {self.blocks[self.rank]}")

    # ---------------------------------------------------------- exchanges
    def _rows(self, names):
        """All-gather the own rows of the named per-row arrays (last axis =
        rows), padded to equal blocks."""
        import torch
        self.e.sync()
        lo, hi = self.blocks[self.rank]
        for name in names:
            a = self.e.array(name)
            shape = a.shape[:-1] + (self.blk,)
            send = torch.zeros(shape, dtype=a.dtype, device=a.device)
            send[..., :hi - lo] = a[..., lo:hi]
            got = self.comm.allgather(send)
            for r, (rl, rh) in enumerate(self.blocks):
                if r != self.rank and rh > rl:
                    a[..., rl:rh] = got[r][..., :rh - rl]
        self.e.sync_torch()

    def _gather_var(self, t):
        """All-gather tensors of different first dimensions (padded to the
        largest); returns the list of each rank's rows."""
        import torch
        n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
        counts = [int(x.item()) for x in self.comm.allgather(n)]
        m = max(1, max(counts))
        pad = torch.zeros((m,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[:t.shape[0]] = t
        got = self.comm.allgather(pad)
        return [g[:c] for g, c in zip(got, counts)]

    def _encounters(self):
        import torch
        own = self.e.own_encounters()           # [n, 2] int32
        allp = torch.cat(self._gather_var(own), 0)
        self.e.import_encounters(allp)

    def _members(self):
        import torch
        rows = self.e.own_members()             # int64 [k]
        q1, v1, hc = self.e.array("q1"), self.e.array("v1"), self.e.array("hcost")
        vals = torch.cat([q1[:, rows], v1[:, rows]], 0).T.contiguous()   # [k, 6]
        g_rows = self._gather_var(rows)
        g_vals = self._gather_var(vals)
        g_hc = self._gather_var(hc[rows].contiguous())
        for r in range(self.world):
            if r == self.rank or g_rows[r].shape[0] == 0:
                continue
            idx = g_rows[r]
            q1[:, idx] = g_vals[r][:, 0:3].T
            v1[:, idx] = g_vals[r][:, 3:6].T
            hc[idx] = g_hc[r]
        self.e.sync_torch()

    # ---------------------------------------------------------- the step
    def step(self, tau: float, nsteps: int) -> None:
        """nsteps steps of size tau (the same call on every rank)."""
        if nsteps < 1:
            return
        e = self.e
        e.phase(QYM_PHASE_OPEN, tau)
        for s in range(nsteps):
            last = int(s == nsteps - 1)
            e.phase(QYM_PHASE_KICK1, tau)
            self._rows(self.ROW_ARRAYS_KICK1)
            e.phase(QYM_PHASE_SEARCH, tau)
            e.phase(QYM_PHASE_KEPLER, tau)
            self._rows(self.ROW_ARRAYS_KEPLER)
            e.phase(QYM_PHASE_REFINE, tau)
            self._encounters()
            e.phase(QYM_PHASE_HERMITE, tau)
            self._members()
            e.phase(QYM_PHASE_KICK2, tau)
            self._rows(self.ROW_ARRAYS_KICK2)
            e.phase(QYM_PHASE_CLOSE, tau, last)


class _CudaArray:
    """A device array of the library exposed to torch without a copy
    (__cuda_array_interface__, version 3)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None, "stream": None}


class GpuEngine:
    """One rank's libqym context on its GPU (qym_split_init, qym_split_phase)."""

    def __init__(self, sim, rank: int, world: int):
        import torch
        from . import lib, _check, qym_split_view
        self.torch = torch
        self.sim = sim
        self.ctx = sim.ctx
        self.L = lib()
        _check(self.L.qym_split_init(self.ctx, rank, world), self.ctx)
        vw = qym_split_view()
        _check(self.L.qym_split_arrays(self.ctx, C.byref(vw)), self.ctx)
        self.rows = int(vw.rows)
        self.own = (int(vw.own_lo), int(vw.own_hi))
        R = self.rows

        def arr(ptr, shape, ts, dtype):
            return torch.as_tensor(_CudaArray(ptr, shape, ts), device="cuda")

        self._arrays = {
            "q": arr(vw.q, (3, R), "<f8", None), "v": arr(vw.v, (3, R), "<f8", None),
            "q1": arr(vw.q1, (3, R), "<f8", None), "v1": arr(vw.v1, (3, R), "<f8", None),
            "rH": arr(vw.rH, (R,), "<f8", None), "amag": arr(vw.amag, (R,), "<f4", None),
            "hcost": arr(vw.hcost, (R,), "<i4", None),
        }
        self._enc = arr(vw.enc, (int(vw.max_enc), 2), "<i4", None)
        self._set_mem = arr(vw.set_mem, (R,), "<i4", None)
        self.stream = torch.cuda.ExternalStream(int(vw.stream or 0))

    def array(self, name):
        return self._arrays[name]

    def phase(self, ph, tau, last=0):
        from . import _check
        _check(self.L.qym_split_phase(self.ctx, ph, float(tau), int(last)), self.ctx)

    def sync(self):
        """The context's work done before torch reads its arrays."""
        self.stream.synchronize()

    def sync_torch(self):
        """torch's writes done before the context's next phase."""
        self.torch.cuda.current_stream().synchronize()

    def own_encounters(self):
        from . import _check
        n = C.c_int64()
        _check(self.L.qym_split_encounter_count(self.ctx, C.byref(n)), self.ctx)
        return self._enc[:n.value].clone()

    def import_encounters(self, pairs):
        from . import _check
        pairs = pairs.to(dtype=self.torch.int32).contiguous()
        self.sync_torch()
        _check(self.L.qym_split_import_encounters(self.ctx, pairs.data_ptr() if len(pairs) else None,
                                                  len(pairs)), self.ctx)
        self.sync()  # the list is read from `pairs`, which dies with this call

    def own_members(self):
        from . import _check
        first, count = C.c_int64(), C.c_int64()
        _check(self.L.qym_split_owned_members(self.ctx, C.byref(first), C.byref(count)), self.ctx)
        f, k = first.value, count.value
        return self._set_mem[f:f + k].to(self.torch.int64)


def split_rows_library(rows: int, rank: int, world: int):
    """The library's blocks (qym_split_rows), for checking split_rows."""
    from . import lib
    lo, hi = C.c_int64(), C.c_int64()
    lib().qym_split_rows(rows, rank, world, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def numpy_blocks(rows: int, world: int):
    return np.array([split_rows(rows, r, world) for r in range(world)], dtype=np.int64)
