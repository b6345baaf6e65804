"""Slab decomposition along z (paper_0809_4730_gb300.slabs), host logic on CPU.

The plan: which slab owns which planes, where the ghost planes and walls
are, who the neighbours are.  The rank transport: two (and three) gloo ranks
on 127.0.0.1, each holding one slab whose populations are tagged by global
plane, direction and position, exchange their faces through the module's
point-to-point exchange; every ghost plane must then hold exactly the
crossing populations of its neighbour's outermost computed plane, and the
FP64 all-reduce of the residual sums must give every rank the grid's record.
The slab handle here is a numpy stand-in for the CUDA context (its pack and
unpack copy the e_z = +-1 rows the library's halo kernels copy).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

# D3Q19 velocities in the ordering of include/glbe.h; the directions that
# cross a z face
E = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
     (1, 1, 0), (-1, 1, 0), (1, -1, 0), (-1, -1, 0), (1, 0, 1), (-1, 0, 1), (1, 0, -1), (-1, 0, -1),
     (0, 1, 1), (0, -1, 1), (0, 1, -1), (0, -1, -1)]
EZ_PLUS = [a for a in range(19) if E[a][2] == 1]
EZ_MINUS = [a for a in range(19) if E[a][2] == -1]


def test_plan_covers_every_plane_once():
    from paper_0809_4730_gb300.slabs import global_planes, plan
    for nz, walls in ((12, (0, 0)), (12, (1, 1)), (7, (1, 1)), (9, (0, 0))):
        for n in range(1, 5):
            sl = plan(nz, n, *walls)
            owned = []
            for s in sl:
                g = global_planes(s, nz)
                own = g[s.ghost_lo: len(g) - s.ghost_hi]
                owned += own
                assert s.nz_local == len(g)
                assert not (s.ghost_lo and s.wall_lo) and not (s.ghost_hi and s.wall_hi)
                if n > 1:
                    # a ghost plane is the neighbour's outermost owned plane
                    if s.ghost_lo:
                        d = sl[s.down]
                        assert g[0] == global_planes(d, nz)[d.nz_local - 1 - d.ghost_hi]
                    if s.ghost_hi:
                        u = sl[s.up]
                        assert g[-1] == global_planes(u, nz)[u.ghost_lo]
            assert sorted(owned) == list(range(nz))
            sizes = [s.z1 - s.z0 - s.wall_lo - s.wall_hi for s in sl]
            assert max(sizes) - min(sizes) <= 1
            if walls == (1, 1):
                assert sl[0].wall_lo == 1 and sl[-1].wall_hi == 1 and sl[0].down is None and sl[-1].up is None
            elif n > 1:
                assert all(s.ghost_lo and s.ghost_hi for s in sl)


def test_plan_rejects_impossible_splits():
    from paper_0809_4730_gb300.slabs import plan
    with pytest.raises(ValueError):
        plan(4, 3, 1, 1)            # 2 computed planes, 3 slabs
    with pytest.raises(ValueError):
        plan(8, 2, 1, 0)            # a wall on one z face only


class _NumpySlab:
    """Stand-in for a slab context: f[a, l, p] (local plane l, position p in
    the plane) tagged 1000 * global plane + 10 * a + p / P; pack copies the
    crossing rows of the outermost computed plane, unpack writes the ghost."""

    def __init__(self, s, nz, P):
        import torch
        from paper_0809_4730_gb300.slabs import global_planes
        self.torch, self.s, self.P = torch, s, P
        g = global_planes(s, nz)
        self.f = np.zeros((19, s.nz_local, P))
        for l, gz in enumerate(g):
            ghost = (l == 0 and s.ghost_lo) or (l == s.nz_local - 1 and s.ghost_hi)
            if not ghost:
                for a in range(19):
                    self.f[a, l] = 1000.0 * gz + 10.0 * a + np.arange(P) / P

    def halo_bytes(self):
        return 5 * self.P * 8

    def new_buffer(self, n):
        return self.torch.zeros(n // 8, dtype=self.torch.float64)

    def pack(self, face, buf):
        l = self.s.nz_local - 2 if face == 1 else 1
        rows = EZ_PLUS if face == 1 else EZ_MINUS
        buf.copy_(self.torch.from_numpy(self.f[rows, l].reshape(-1).copy()))

    def unpack(self, face, buf):
        l = 0 if face == 0 else self.s.nz_local - 1
        rows = EZ_PLUS if face == 0 else EZ_MINUS
        self.f[rows, l] = buf.numpy().reshape(5, self.P)

    def sync(self):
        pass

    def step(self, n):
        pass

    def residual(self):
        from paper_0809_4730_gb300.glbe import glbe_residual_info
        r = glbe_residual_info()
        k = self.s.k
        r.t, r.num, r.den, r.mass = 40, 1e-10 * (k + 1), 2.0 * (k + 1), 100.0 + k
        r.momentum[0], r.momentum[1], r.momentum[2] = 0.5 * k, -1.0, 2.0
        return r

    def reduce_device(self):
        return "cpu"


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, nz, walls, out):
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    from paper_0809_4730_gb300.slabs import RankSlab, global_planes, plan
    dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=20))
    try:
        P = 6
        sl = plan(nz, ws, *walls)
        op = _NumpySlab(sl[rank], nz, P)
        R = RankSlab(sl, rank, op)
        R.step(1)
        s = sl[rank]
        g = global_planes(s, nz)
        ok = True
        for face, l, rows in ((0, 0, EZ_PLUS), (1, s.nz_local - 1, EZ_MINUS)):
            if (s.ghost_lo if face == 0 else s.ghost_hi):
                want = np.array([[1000.0 * g[l] + 10.0 * a + p / P for p in range(P)] for a in rows])
                ok = ok and np.array_equal(op.f[rows, l], want)
        rec = R.residual()
        out.put((rank, "ok", ok, rec.t, rec.num, rec.den, rec.r, rec.mass, tuple(rec.momentum[:])))
    except Exception as e:
        out.put((rank, "error", repr(e), 0, 0, 0, 0, 0, ()))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


@pytest.mark.parametrize("ws,nz,walls", [(2, 10, (0, 0)), (2, 9, (1, 1)), (3, 11, (1, 1)), (3, 9, (0, 0))])
def test_rank_exchange_fills_every_ghost_plane(ws, nz, walls):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, nz, walls, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    res = {}
    while not q.empty():
        item = q.get()
        res[item[0]] = item[1:]
    assert sorted(res) == list(range(ws)), res
    num = sum(1e-10 * (k + 1) for k in range(ws))
    den = sum(2.0 * (k + 1) for k in range(ws))
    for r in range(ws):
        status, ok, t, rn, rd, rr, rm, mom = res[r]
        assert status == "ok", ok
        assert ok, f"rank {r}: a ghost plane does not hold its neighbour's crossing populations"
        assert t == 40 and rn == pytest.approx(num, rel=1e-15) and rd == pytest.approx(den, rel=1e-15)
        assert rr == pytest.approx(np.sqrt(num / den), rel=1e-14)
        assert rm == pytest.approx(sum(100.0 + k for k in range(ws)), rel=1e-15)
        assert mom[0] == pytest.approx(sum(0.5 * k for k in range(ws))) and mom[1] == -1.0 * ws
