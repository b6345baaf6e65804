"""Slab decomposition along z on one GPU: 2 and 3 slabs (contexts with
ghost planes) exchanging their faces after every step through
glbe_halo_pack / glbe_halo_unpack must march bit for bit like the whole grid
-- every node's update reads the same populations -- and their combined
residual record must be the grid's (the FP32 per-block sums group other
nodes, hence the relative bound on r)."""
import numpy as np
import pytest

from gpu_common import require_cuda

pytestmark = pytest.mark.gpu


def _setup(storage, mhd, zwalls, nslabs, nx=16, ny=10, nz=13):
    from paper_0809_4730_gb300.glbe import Solver
    from paper_0809_4730_gb300.inputs import perturbation, random_force
    from paper_0809_4730_gb300.slabs import LocalSlabs, SolverSlab, global_planes, plan, slab_params
    torch = require_cuda()
    w = int(zwalls)
    kw = dict(wall_lo=(0, 1, w), wall_hi=(0, 1, w), gamma=0.3, nu=0.03, storage=storage, force_field=3)
    if mhd:
        kw.update(induction=1, gamma_m=0.3, eta=0.03, chi=0.2, mu=1.0, B0=(0.0, 0.02, 0.01))
    W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    df = perturbation(19, nx, ny, nz, 2e-3, seed=4) * W[:, None, None, None]
    dg = perturbation(21, nx, ny, nz, 1e-4, seed=5) if mhd else None
    FL = perturbation(3, nx, ny, nz, 1e-6, seed=6) if mhd else None
    F = random_force(nx, ny, nz, 2e-5, seed=7)
    dev = lambda a, q: torch.tensor(a.reshape(q, -1), dtype=torch.float32, device="cuda")

    G = Solver(nx, ny, nz, **kw)
    G.set_force(dev(F, 3))
    G.set_state(dev(df, 19), None if dg is None else dev(dg, 21), None if FL is None else dev(FL, 3), t=0)

    slabs = plan(nz, nslabs, w, w)
    ops = []
    for s in slabs:
        zs = global_planes(s, nz)
        cut = lambda a: np.ascontiguousarray(a[:, zs])
        S = Solver(nx, ny, s.nz_local, **slab_params(kw, s))
        S.set_force(dev(cut(F), 3))
        S.set_state(dev(cut(df), 19), None if dg is None else dev(cut(dg), 21),
                    None if FL is None else dev(cut(FL), 3), t=0)
        ops.append(SolverSlab(S))
    return G, LocalSlabs(slabs, ops), slabs


@pytest.mark.parametrize("nslabs", [2, 3])
@pytest.mark.parametrize("zwalls", [False, True])
@pytest.mark.parametrize("storage,mhd", [("f32", False), ("bf16", False), ("f32c", False), ("f32", True),
                                         ("bf16", True), ("f32c", True)])
def test_slabs_march_bit_for_bit_like_the_grid(storage, mhd, zwalls, nslabs):
    from paper_0809_4730_gb300.slabs import global_planes
    G, L, slabs = _setup(storage, mhd, zwalls, nslabs)
    nz = G.params.nz
    G.step(23)
    L.step(23)
    want = [a for a in G.get_state()]
    G.sync()
    for s, o in zip(slabs, L.ops):
        got = o.G.get_state()
        o.G.sync()
        zs = global_planes(s, nz)
        own = slice(s.ghost_lo, s.nz_local - s.ghost_hi)
        for a, b in zip(got, want):
            if a is None:
                continue
            q = a.shape[0]
            a = a.reshape(q, s.nz_local, -1)[:, own].cpu().numpy()
            b = b.reshape(q, nz, -1)[:, zs[own]].cpu().numpy()
            assert np.array_equal(a, b), (s, q)
    rg = G.residual()
    rs = L.residual()
    assert rs.t == rg.t == 20
    assert abs(rs.r - rg.r) <= 1e-6 * rg.r
    assert abs(rs.mass - rg.mass) <= 1e-12 * rg.mass
    assert np.allclose(rs.momentum[:], rg.momentum[:], rtol=1e-5, atol=1e-12)


def test_halo_entry_points_reject_a_face_without_ghost_plane():
    from paper_0809_4730_gb300.glbe import GLBE_ERR_STATE, GlbeError, Solver, glbe_halo_bytes, glbe_halo_pack
    torch = require_cuda()
    G = Solver(8, 6, 5, wall_lo=(0, 1, 1), wall_hi=(0, 1, 0), ghost_hi=1, nu=0.05)
    buf = torch.empty(glbe_halo_bytes(G.ctx), dtype=torch.uint8, device="cuda")
    assert buf.numel() == 5 * 8 * 6 * 4
    glbe_halo_pack(G.ctx, 1, buf)
    with pytest.raises(GlbeError) as ei:
        glbe_halo_pack(G.ctx, 0, buf)
    assert ei.value.status == GLBE_ERR_STATE
    G.close()
