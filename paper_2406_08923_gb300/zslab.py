"""Z-slab decomposition of one periodic 3D grid over P ranks (one GPU per rank).

The paper runs every workload on a single device (Sec. 5.1); this module is the multi-GPU
form of the same computation.  Rank p owns the planes [z0, z1) of the grid (a balanced split,
every slab at least r planes thick) as a plan with boundary mode STENCIL_BC_PERIODIC_XY: the
library keeps x and y periodic, and before every pass the r halo planes below and above the
slab are filled with the neighbouring slabs' edge planes (periodic along z, so rank 0's lower
neighbour is rank P-1):

  * my lowest r interior planes  -> the upper z halo of rank p-1,
  * my highest r interior planes -> the lower z halo of rank p+1.

A heat step (Eqs. 4-7) is one pass, so one exchange per Euler step; an MHD RK3 step (Sec. 3.3,
Eqs. A1-A4) is three passes, so one exchange per substep, of all 8 fields.  Whole padded planes
are sent (the x/y halos ride along).  The per-field reductions combine with one all-reduce:
sum and sum of squares (and the mass) add, max |f| takes the maximum.

Transports:
  * DistTransport -- torch.distributed point-to-point (NCCL between GPUs, gloo for CPU
    tensors), all sends and receives of one exchange in one batch.
  * LocalSlabs    -- all P slabs in one process (e.g. on one GPU), the exchange as device
    copies in stream order; it exercises the same plane bookkeeping and the same kernels.

Only plane arithmetic and data movement live here; every stencil pass runs in the library.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import _lib as L


def slab_bounds(nz: int, nranks: int, rank: int, r: int = 3) -> tuple[int, int]:
    """[z0, z1) of `rank`'s slab: nz planes split as evenly as possible (the first nz % nranks
    slabs one plane thicker).  Every slab must hold at least r planes, so that its halo comes
    from its two neighbours only."""
    if not 0 <= rank < nranks:
        raise ValueError(f"rank {rank} outside 0..{nranks - 1}")
    base, extra = divmod(nz, nranks)
    if base < r:
        raise ValueError(f"{nz} planes over {nranks} ranks leaves slabs thinner than the radius {r}")
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


@dataclass(frozen=True)
class SlabPlanes:
    """Plane ranges of one slab's padded field (z-major, planes of padded[0] * padded[1])."""

    padded: tuple
    origin_z: int
    nz: int
    r: int

    @property
    def plane_elems(self) -> int:
        return int(self.padded[0]) * int(self.padded[1])

    def block(self, t, start: int):
        """The r consecutive padded planes of flat field `t` from plane index `start`."""
        return t.view(int(self.padded[2]), self.plane_elems)[start:start + self.r]

    def lower_halo(self, t):
        return self.block(t, self.origin_z - self.r)

    def upper_halo(self, t):
        return self.block(t, self.origin_z + self.nz)

    def lowest_interior(self, t):
        return self.block(t, self.origin_z)

    def highest_interior(self, t):
        return self.block(t, self.origin_z + self.nz - self.r)


class DistTransport:
    """Halo exchange between ranks with torch.distributed point-to-point operations.

    Operations are issued in an order that pairs up the same way for NCCL (which matches a
    pair's messages in issue order) and for gloo (which matches tags): first the two sends
    (to the lower neighbour, then to the upper), then the two receives (from the upper
    neighbour, then from the lower).  With two ranks both neighbours are the same process and
    this order still pairs each send with the right halo."""

    def __init__(self, rank: int, nranks: int, group=None):
        self.rank, self.nranks, self.group = rank, nranks, group

    def exchange(self, planes: SlabPlanes, fields):
        import torch.distributed as dist
        if self.nranks == 1:
            for t in fields:
                planes.lower_halo(t).copy_(planes.highest_interior(t))
                planes.upper_halo(t).copy_(planes.lowest_interior(t))
            return
        down = (self.rank - 1) % self.nranks
        up = (self.rank + 1) % self.nranks
        # plane blocks are contiguous slices of the z-major field: sent and received in place
        ops = []
        for q, t in enumerate(fields):
            ops.append(dist.P2POp(dist.isend, planes.lowest_interior(t), down, self.group, tag=2 * q))
            ops.append(dist.P2POp(dist.isend, planes.highest_interior(t), up, self.group, tag=2 * q + 1))
        for q, t in enumerate(fields):
            ops.append(dist.P2POp(dist.irecv, planes.upper_halo(t), up, self.group, tag=2 * q))
            ops.append(dist.P2POp(dist.irecv, planes.lower_halo(t), down, self.group, tag=2 * q + 1))
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def allreduce_norms(self, norms, nfields: int):
        """Combine per-slab [sum, sumsq, max|f|] x nfields (+ mass) into whole-grid values."""
        import torch
        import torch.distributed as dist
        if self.nranks == 1:
            return norms
        t = torch.as_tensor(norms, dtype=torch.float64)
        add_idx = [3 * q + c for q in range(nfields) for c in (0, 1)] + list(range(3 * nfields, t.numel()))
        max_idx = [3 * q + 2 for q in range(nfields)]
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        s = t[add_idx].to(dev)
        m = t[max_idx].to(dev)
        dist.all_reduce(s, op=dist.ReduceOp.SUM, group=self.group)
        dist.all_reduce(m, op=dist.ReduceOp.MAX, group=self.group)
        out = t.clone()
        out[add_idx] = s.cpu()
        out[max_idx] = m.cpu()
        return out.numpy()


def _slab_plan(kind, dims, nz_local, storage, params, r):
    nx, ny, _ = dims
    if kind == L.STENCIL_MHD8:
        compute = L.STENCIL_F64 if storage == L.STENCIL_F64 else L.STENCIL_F32
        return L.Plan(3, (nx, ny, nz_local), 3, 8, L.STENCIL_BC_PERIODIC_XY, L.STENCIL_MHD8, storage, compute,
                      params=params)
    return L.Plan(3, (nx, ny, nz_local), r, 1, L.STENCIL_BC_PERIODIC_XY, L.STENCIL_DIFFUSION, storage, storage,
                  params=params)


class ZSlabPlan:
    """This rank's slab of a grid of interior extents dims = (nx, ny, nz), decomposed along z.

    kind: STENCIL_DIFFUSION (radius r, F64 or F32) or STENCIL_MHD8 (F64, F32 or BF16 storage).
    Fields are allocated with alloc() in the slab plan's padded layout; upload() takes the
    whole grid's interior (nz, ny, nx) arrays and keeps this slab's planes."""

    def __init__(self, kind, dims, storage, params, rank, nranks, transport=None, r=3):
        self.kind, self.dims, self.rank, self.nranks = kind, tuple(dims), rank, nranks
        self.r = 3 if kind == L.STENCIL_MHD8 else r
        self.z0, self.z1 = slab_bounds(dims[2], nranks, rank, self.r)
        self.plan = _slab_plan(kind, dims, self.z1 - self.z0, storage, params, self.r)
        self.planes = SlabPlanes(self.plan.padded, self.plan.origin[2], self.z1 - self.z0, self.r)
        self.transport = transport or DistTransport(rank, nranks)

    def alloc(self, device="cuda"):
        return self.plan.alloc(device)

    def upload(self, fields, whole_interiors):
        self.plan.upload(fields, [a[self.z0:self.z1] for a in whole_interiors])

    def download(self, fields):
        return self.plan.download(fields)

    def exchange(self, fields):
        self.transport.exchange(self.planes, fields)

    def step(self, fin, fout, nsteps, stream=None):
        """nsteps Euler steps (DIFFUSION) or RK3 steps (MHD8), each pass preceded by a z-halo
        exchange; the result ends in fout and fin's interior is preserved."""
        if getattr(self, "_tmp", None) is None:
            self._tmp = self.plan.alloc()
        tmp = self._tmp
        passes = [(s % 3) for s in range(3 * nsteps)] if self.kind == L.STENCIL_MHD8 else [0] * nsteps
        if not passes:
            for d, s in zip(fout, fin):
                d.copy_(s)
            return
        src = fin
        for i, sub in enumerate(passes):
            dst = fout if (len(passes) - 1 - i) % 2 == 0 else tmp
            self.exchange(src)
            if self.kind == L.STENCIL_MHD8:
                self.plan.substep(src, dst, sub, stream)
            else:
                self.plan.step(src, dst, 1, stream)
            src = dst

    def norms(self, fields):
        """Whole-grid [sum, sumsq, max|f|] per field (+ MHD mass), all-reduced over the ranks."""
        return self.transport.allreduce_norms(self.plan.norms(fields), self.plan.nfields)


class LocalSlabs:
    """All P slabs of one grid in one process, on one device: the decomposition without a
    second GPU.  The halo exchange is a device copy per block, in stream order; passes run
    slab after slab.  Used to check the decomposition against the single-domain path."""

    def __init__(self, kind, dims, storage, params, nranks, r=3):
        self.kind, self.nranks = kind, nranks
        self.slabs = [ZSlabPlan(kind, dims, storage, params, p, nranks, transport=self, r=r) for p in range(nranks)]
        self._fields = None

    def alloc(self):
        return [s.alloc() for s in self.slabs]

    def upload(self, fields, whole):
        for s, f in zip(self.slabs, fields):
            s.upload(f, whole)

    def download(self, fields):
        import numpy as np
        return np.concatenate([s.download(f) for s, f in zip(self.slabs, fields)], axis=1)

    def exchange_all(self, fields):
        for p, s in enumerate(self.slabs):
            lo_nb, hi_nb = self.slabs[(p - 1) % self.nranks], self.slabs[(p + 1) % self.nranks]
            flo, fhi = fields[(p - 1) % self.nranks], fields[(p + 1) % self.nranks]
            for q, t in enumerate(fields[p]):
                s.planes.lower_halo(t).copy_(lo_nb.planes.highest_interior(flo[q]))
                s.planes.upper_halo(t).copy_(hi_nb.planes.lowest_interior(fhi[q]))

    def exchange(self, planes, fields):  # slab-level calls are driven by step() below
        raise RuntimeError("LocalSlabs exchanges all slabs at once; call LocalSlabs.step")

    def step(self, fin, fout, nsteps, stream=None):
        kind = self.kind
        if getattr(self, "_tmp", None) is None:
            self._tmp = [s.alloc() for s in self.slabs]
        tmp = self._tmp
        passes = [(k % 3) for k in range(3 * nsteps)] if kind == L.STENCIL_MHD8 else [0] * nsteps
        src = fin
        for i, sub in enumerate(passes):
            dst = fout if (len(passes) - 1 - i) % 2 == 0 else tmp
            self.exchange_all(src)
            for p, s in enumerate(self.slabs):
                if kind == L.STENCIL_MHD8:
                    s.plan.substep(src[p], dst[p], sub, stream)
                else:
                    s.plan.step(src[p], dst[p], 1, stream)
            src = dst

    def norms(self, fields):
        import numpy as np
        per = [s.plan.norms(f) for s, f in zip(self.slabs, fields)]
        nf = self.slabs[0].plan.nfields
        out = np.sum(per, axis=0)
        for q in range(nf):
            out[3 * q + 2] = max(x[3 * q + 2] for x in per)
        return out
