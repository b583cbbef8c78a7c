"""One grid decomposed along z into slabs, one context per slab.

The C ABI (bfvm_create_slab, bfvm_slab_forward / _backward / _finish) runs a
step of one slab in three calls; between them every slab's one value per z
line and substrate is gathered, in slab order.  This module holds the host
side of that: the partition of the z layers, the cells of each slab, the
gathers, and two ways to step a decomposed grid:

* ``step_together(slabs, n)``: all slabs of the grid in this process, on one
  device (the gathers are a stack of the slabs' send buffers);
* ``step_distributed(slab, n)``: one slab per rank of the default
  torch.distributed group, rank r holding slab r (the gathers are
  all-gathers: NCCL on device buffers, or gloo through host copies).

The arithmetic of the step is the library's; this module only moves the
gathered values between the calls.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from . import bfvm


def partition(nz: int, n_slabs: int) -> List[int]:
    """z_starts of n_slabs slabs of nearly equal depth (the first nz % n
    slabs one layer deeper): slab j holds layers [z[j], z[j+1])."""
    if not (1 <= n_slabs <= nz):
        raise ValueError(f"need 1 <= n_slabs <= nz, got {n_slabs} slabs of {nz} layers")
    base, extra = divmod(nz, n_slabs)
    z = [0]
    for j in range(n_slabs):
        z.append(z[-1] + base + (1 if j < extra else 0))
    return z


def cell_layers(pos_z, dx: float, nz: int) -> np.ndarray:
    """Global voxel layer of each cell: min(floor(p_z / dx), nz - 1), the
    binning every context applies (FP64 division on both sides)."""
    q = np.floor(np.asarray(pos_z, dtype=np.float64) / float(dx)).astype(np.int64)
    return np.clip(q, 0, nz - 1)


def cell_slabs(pos_z, dx: float, z_starts: Sequence[int]) -> np.ndarray:
    """Slab index of each cell: the slab holding its voxel layer."""
    zs = np.asarray(z_starts, dtype=np.int64)
    return np.searchsorted(zs, cell_layers(pos_z, dx, int(zs[-1])), side="right") - 1


class Slab:
    """The context of one z-slab; field and cells in the slab's own part of
    the grid (cells in grid coordinates)."""

    def __init__(self, nx, ny, z_starts, slab, dx, dt, D, lam, bc_kind, bc_value, stream=None,
                 device=None):
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.z_starts = [int(v) for v in z_starts]
        self.slab = int(slab)
        self.n_slabs = len(self.z_starts) - 1
        self.nz = self.z_starts[slab + 1] - self.z_starts[slab]
        self.shape = (len(D), self.nz, ny, nx)
        self.handle = bfvm.bfvm_create_slab(nx, ny, self.z_starts, slab, dx, dt, D, lam, bc_kind,
                                            bc_value, self.stream)
        self.send = torch.zeros((len(D), ny, nx), dtype=torch.float64, device=self.device)

    @classmethod
    def from_problem(cls, p, z_starts, slab, stream=None):
        """Slab `slab` of a whole-grid Problem: its layers of the initial
        field and the cells whose voxel lies in it."""
        import torch
        s = cls(p.nx, p.ny, z_starts, slab, p.dx, p.dt, p.D, p.lam, p.bc_kind, p.bc_value, stream)
        z0, z1 = z_starts[slab], z_starts[slab + 1]
        s.set_density(torch.as_tensor(np.ascontiguousarray(p.rho0[:, z0:z1]), dtype=torch.float64,
                                      device=s.device))
        if p.n_cells:
            mine = np.nonzero(cell_slabs(p.pos[:, 2], p.dx, z_starts) == slab)[0]
            if mine.size:
                s.set_cells(*[torch.as_tensor(np.ascontiguousarray(a[mine]), dtype=torch.float64,
                                              device=s.device)
                              for a in (p.pos, p.vol, p.S, p.U, p.rho_star)])
        return s

    def set_density(self, rho):
        bfvm.bfvm_set_density(self.handle, rho)

    def get_density(self):
        import torch
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        bfvm.bfvm_get_density(self.handle, out)
        return out

    def set_cells(self, pos, vol, S, U, rho_star):
        bfvm.bfvm_set_cells(self.handle, pos, vol, S, U, rho_star)

    def forward(self):
        bfvm.bfvm_slab_forward(self.handle, self.send)

    def backward(self, gathered):
        bfvm.bfvm_slab_backward(self.handle, gathered, self.send)

    def finish(self, gathered):
        bfvm.bfvm_slab_finish(self.handle, gathered)

    def close(self):
        if getattr(self, "handle", None) is not None:
            bfvm.bfvm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_together(slabs: Sequence[Slab], n_steps: int = 1) -> None:
    """n steps of a grid whose slabs all live in this process (one stream:
    every slab's calls and the stacks between them are ordered on it)."""
    import torch
    for _ in range(int(n_steps)):
        for s in slabs:
            s.forward()
        gathered = torch.stack([s.send for s in slabs])
        for s in slabs:
            s.backward(gathered)
        gathered = torch.stack([s.send for s in slabs])
        for s in slabs:
            s.finish(gathered)


def all_gather_slabs(send, group=None):
    """(world, *send.shape) of every rank's send buffer, in rank order, on
    send's device: NCCL gathers device buffers directly; other backends
    (gloo) gather host copies."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = torch.empty((world,) + tuple(send.shape), dtype=send.dtype, device=send.device)
    if dist.get_backend(group) == "nccl":
        dist.all_gather_into_tensor(out, send, group=group)
        return out
    host = send.detach().cpu()
    parts = [torch.empty_like(host) for _ in range(world)]
    dist.all_gather(parts, host, group=group)
    out.copy_(torch.stack(parts))
    return out


def step_distributed(slab: Slab, n_steps: int = 1, group=None, gather=all_gather_slabs) -> None:
    """n steps of this rank's slab of a grid decomposed one slab per rank
    (rank r holds slab r)."""
    import torch.distributed as dist
    if dist.get_world_size(group) != slab.n_slabs or dist.get_rank(group) != slab.slab:
        raise ValueError("rank r of the group must hold slab r of n_slabs == world size")
    for _ in range(int(n_steps)):
        slab.forward()
        slab.backward(gather(slab.send, group))
        slab.finish(gather(slab.send, group))
