"""Slab decomposition of a grid along z: host-side orchestration of the C-ABI.

The time step is local except nearest-neighbour streaming (Eqs. pstreaming,
mstreaming), so a grid splits into slabs of z planes, each a context with
ghost planes (``ghost_lo`` / ``ghost_hi`` of glbe_params).  After every step
the populations that cross a slab face -- the 5 D3Q19 directions with
e_z = +-1 and, with induction, the D3Q7 direction e_z = +-1 of each of the 3
components -- are packed on one side (glbe_halo_pack), moved to the
neighbour, and unpacked into its ghost plane (glbe_halo_unpack).  Every 10
levels each slab's residual record holds its FP64 sums; the grid's record is
their sum (an FP64 all-reduce across ranks, then glbe_residual_combine).
The lagged Lorentz force is local: nothing else crosses a face.

This module holds no arithmetic of the method: it decides which slab owns
which planes, which buffer goes to which neighbour, and when.  Two transports:

- ``LocalSlabs``: all slabs in this process (on one device or several),
  each face moved by the device copy of its unpack from the neighbour's
  packed buffer;
- ``RankSlab``: one slab per rank of a torch.distributed process group
  (NCCL between GPUs, gloo on CPU), faces moved by point-to-point
  send/receive, the residual sums by an all-reduce.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Slab:
    """Slab k of a grid: global planes [z0, z1) computed or on a wall, with a
    ghost plane below (ghost_lo) and/or above (ghost_hi).  Local plane l
    holds global plane z0 - ghost_lo + l (taken modulo nz across a periodic
    z axis)."""
    k: int
    z0: int
    z1: int
    ghost_lo: int
    ghost_hi: int
    wall_lo: int
    wall_hi: int
    down: int | None      # slab below (None: a wall)
    up: int | None        # slab above

    @property
    def nz_local(self) -> int:
        return self.z1 - self.z0 + self.ghost_lo + self.ghost_hi

    def local_of(self, z: int) -> int:
        return z - self.z0 + self.ghost_lo


def plan(nz: int, nslabs: int, wall_lo_z: int = 0, wall_hi_z: int = 0) -> list[Slab]:
    """Splits the nz planes of a grid into nslabs contiguous slabs of nearly
    equal size.  With walls on z the wall planes stay in the first and last
    slab (as walls); without, z is periodic and every slab has two ghost
    planes.  Every slab keeps at least one computed plane."""
    if nslabs < 1:
        raise ValueError("nslabs must be >= 1")
    computed = nz - wall_lo_z - wall_hi_z
    if computed < nslabs:
        raise ValueError(f"{computed} computed planes cannot make {nslabs} slabs")
    periodic = not wall_lo_z and not wall_hi_z
    if bool(wall_lo_z) != bool(wall_hi_z):
        raise ValueError("a slab plan needs walls on both z faces or on none")
    base, extra = divmod(computed, nslabs)
    out, z = [], wall_lo_z
    for k in range(nslabs):
        n = base + (1 if k < extra else 0)
        z0, z1 = z, z + n
        z = z1
        first, last = k == 0, k == nslabs - 1
        wl = int(first and bool(wall_lo_z))
        wh = int(last and bool(wall_hi_z))
        if wl:
            z0 -= 1                         # the wall plane belongs to the first slab
        if wh:
            z1 += 1
        if nslabs == 1 and not periodic:
            gl = gh = 0
        else:
            gl, gh = int(not wl), int(not wh)
        if nslabs == 1 and periodic:
            gl = gh = 0                     # the whole periodic grid: no ghost planes
        down = None if wl else (k - 1) % nslabs
        up = None if wh else (k + 1) % nslabs
        if nslabs == 1:
            down = up = None
        out.append(Slab(k, z0, z1, gl, gh, wl, wh, down, up))
    return out


def slab_params(kw: dict, s: Slab) -> dict:
    """Keyword parameters of slab s from the grid's (walls on x, y kept;
    the z walls and ghost planes of the slab)."""
    out = dict(kw)
    wl = list(kw.get("wall_lo", (0, 0, 0)))
    wh = list(kw.get("wall_hi", (0, 0, 0)))
    wl[2], wh[2] = s.wall_lo, s.wall_hi
    out.update(wall_lo=tuple(wl), wall_hi=tuple(wh), ghost_lo=s.ghost_lo, ghost_hi=s.ghost_hi)
    return out


def global_planes(s: Slab, nz: int) -> list[int]:
    """Global plane index of every local plane of slab s (ghost planes
    included, wrapped across a periodic z axis)."""
    return [(s.z0 - s.ghost_lo + l) % nz for l in range(s.nz_local)]


# ---------------------------------------------------------------------------
# Transports
# ---------------------------------------------------------------------------
class LocalSlabs:
    """All slabs of a grid in this process.  ``ops[k]`` is slab k's handle
    with ``step(n)``, ``halo_bytes()``, ``pack(face, buf)``,
    ``unpack(face, buf)``, ``residual()`` and ``new_buffer(nbytes)``."""

    def __init__(self, slabs: list[Slab], ops):
        self.slabs, self.ops = slabs, ops
        self.bufs = {}
        for s, o in zip(slabs, ops):
            n = o.halo_bytes()
            for face, has in ((0, s.ghost_lo), (1, s.ghost_hi)):
                if has:
                    self.bufs[(s.k, face)] = o.new_buffer(n)

    def exchange(self):
        """Moves every face: slab k's face-1 pack into its upper neighbour's
        low ghost plane, its face-0 pack into its lower neighbour's high one.
        All packs are taken before any unpack (with one periodic slab its own
        ghost planes are its neighbours')."""
        for s, o in zip(self.slabs, self.ops):
            if s.up is not None:
                o.pack(1, self.bufs[(s.k, 1)])
            if s.down is not None:
                o.pack(0, self.bufs[(s.k, 0)])
        for s, o in zip(self.slabs, self.ops):
            if s.up is not None:
                self.ops[s.up].unpack(0, self.bufs[(s.k, 1)])
            if s.down is not None:
                self.ops[s.down].unpack(1, self.bufs[(s.k, 0)])

    def step(self, n: int):
        for _ in range(n):
            for o in self.ops:
                o.step(1)
            self.exchange()

    def residual(self):
        from .glbe import glbe_residual_combine
        return glbe_residual_combine([o.residual() for o in self.ops])


class RankSlab:
    """Slab ``rank`` of a grid whose slabs are the ranks of the default
    torch.distributed process group (rank k holds slab k).  ``op`` is the
    slab's handle as for LocalSlabs; buffers live on ``op``'s device (NCCL)
    or on the CPU (gloo)."""

    def __init__(self, slabs: list[Slab], rank: int, op):
        import torch.distributed as dist
        self.dist = dist
        if dist.get_world_size() != len(slabs):
            raise ValueError("one slab per rank")
        self.s, self.op = slabs[rank], op
        n = op.halo_bytes()
        self.send = {f: op.new_buffer(n) for f, h in ((0, self.s.ghost_lo), (1, self.s.ghost_hi)) if h}
        self.recv = {f: op.new_buffer(n) for f in self.send}

    def exchange(self):
        """Packs both faces, then one batch of point-to-point transfers in
        two phases: upward (the face-1 pack to the upper neighbour; the lower
        neighbour's face-1 pack into the low ghost plane), then downward.
        Two slabs on a periodic axis are each other's upper and lower
        neighbour: the fixed phase order (and the tags, where the transport
        uses them) keeps the two transfers of one pair apart."""
        dist, s = self.dist, self.s
        for f in self.send:
            self.op.pack(f, self.send[f])
        self.op.sync()
        UP, DOWN = 1, 2
        ops = []
        if s.up is not None:
            ops.append(dist.P2POp(dist.isend, self.send[1], s.up, tag=UP))
        if s.down is not None:
            ops.append(dist.P2POp(dist.irecv, self.recv[0], s.down, tag=UP))
        if s.down is not None:
            ops.append(dist.P2POp(dist.isend, self.send[0], s.down, tag=DOWN))
        if s.up is not None:
            ops.append(dist.P2POp(dist.irecv, self.recv[1], s.up, tag=DOWN))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        # face 0 takes what the lower neighbour sent up, face 1 what came down
        for f in self.recv:
            self.op.unpack(f, self.recv[f])

    def step(self, n: int):
        for _ in range(n):
            self.op.step(1)
            self.exchange()

    def residual(self):
        """The grid's record: the slab records' FP64 sums added over all
        ranks (all-reduce), r formed by glbe_residual_combine."""
        import torch
        from .glbe import glbe_residual_combine, glbe_residual_info
        mine = self.op.residual()
        dev = self.op.reduce_device()
        v = torch.tensor([mine.num, mine.den, mine.mass, *mine.momentum[:], float(mine.nonfinite), float(mine.t)],
                         dtype=torch.float64, device=dev)
        tmax = v[-1:].clone()
        self.dist.all_reduce(v, op=self.dist.ReduceOp.SUM)
        self.dist.all_reduce(tmax, op=self.dist.ReduceOp.MAX)
        world = self.dist.get_world_size()
        tot = glbe_residual_info()
        tot.t = mine.t
        tot.num, tot.den, tot.mass = float(v[0]), float(v[1]), float(v[2])
        for k in range(3):
            tot.momentum[k] = float(v[3 + k])
        tot.nonfinite = int(v[6])
        if int(tmax.item()) * world != int(v[7].item()):
            raise RuntimeError("slabs report residual records of different levels")
        return glbe_residual_combine([tot])


class SolverSlab:
    """Slab handle over a CUDA context (paper_0809_4730_gb300.glbe.Solver)."""

    def __init__(self, solver):
        self.G = solver

    def step(self, n: int):
        self.G.step(n)

    def halo_bytes(self) -> int:
        from .glbe import glbe_halo_bytes
        return glbe_halo_bytes(self.G.ctx)

    def new_buffer(self, nbytes: int):
        return self.G.torch.empty(nbytes, dtype=self.G.torch.uint8, device=self.G.device)

    def pack(self, face: int, buf):
        from .glbe import glbe_halo_pack
        glbe_halo_pack(self.G.ctx, face, buf)

    def unpack(self, face: int, buf):
        from .glbe import glbe_halo_unpack
        glbe_halo_unpack(self.G.ctx, face, buf)

    def sync(self):
        self.G.sync()

    def residual(self):
        return self.G.residual()

    def reduce_device(self):
        return self.G.device
