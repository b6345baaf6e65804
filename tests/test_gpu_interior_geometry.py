"""Geometries at the edge of the interior fast path, against the FP64 oracle.

A node takes the interior gather (fixed offsets per direction, no geometry)
when its neighbours are fluid and no source crosses a y or z seam; on an x
axis without walls every x qualifies, the sources across the x seam being
moved by nx.  These cases put the seam on every node (nx = 1, where the
source across the seam is the node itself, and nx = 2, 3), leave x walled
(no interior node on x = 0 or nx - 1) or walled on one side only (x = nx - 1
wraps onto a wall plane), and make y and z periodic (their seam rows take the
general gather while the x seam stays on the interior one).  The forward step
is compared after 13 steps at the FP32 bar of test_gpu_parity.py (3e-5 of the
largest deviation); the reverse step through the unrolled adjoint at the bar
of test_gpu_adjoint.py (5e-5 of max |dQ/dF| for 60 steps).
"""
import numpy as np
import pytest

from gpu_common import W19, W7, gpu_state, make_pair, oracle_state_dev, push_oracle_state, rel_linf

pytestmark = pytest.mark.gpu

# (nx, ny, nz, wall_lo, wall_hi)
GEOMETRIES = [
    (1, 8, 7, (0, 1, 1), (0, 1, 1)),
    (2, 8, 7, (0, 1, 1), (0, 1, 1)),
    (3, 7, 8, (0, 1, 1), (0, 1, 0)),
    (9, 6, 7, (0, 0, 0), (0, 0, 0)),     # fully periodic box
    (9, 7, 6, (1, 0, 1), (1, 0, 1)),     # walls on x and z, y periodic
    (9, 7, 7, (1, 1, 1), (0, 1, 1)),     # one x wall: x = nx - 1 wraps onto it
]


def _perturb(S, seed, scale=2e-3):
    from paper_0809_4730_gb300.inputs import perturbation
    cfg = S.cfg
    S.f += perturbation(19, cfg.nx, cfg.ny, cfg.nz, scale, seed).reshape(19, -1).T * W19[None, :]
    if cfg.induction:
        q = perturbation(21, cfg.nx, cfg.ny, cfg.nz, scale * 0.05, seed + 1).reshape(21, -1).T
        S.g += q.reshape(cfg.N, 3, 7) * W7[None, None, :]
        S.FL[:] = perturbation(3, cfg.nx, cfg.ny, cfg.nz, 1e-6, seed + 2).reshape(3, -1).T


@pytest.mark.parametrize("geom", GEOMETRIES, ids=[f"{g[0]}x{g[1]}x{g[2]}-lo{g[3]}-hi{g[4]}" for g in GEOMETRIES])
@pytest.mark.parametrize("mhd", [False, True])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_step_parity_at_interior_edges(orc, geom, mhd, storage):
    from paper_0809_4730_gb300.inputs import random_force
    nx, ny, nz, lo, hi = geom
    kw = dict(wall_lo=lo, wall_hi=hi, gamma=0.3, nu=0.02, F=(2e-5, -1e-5, 5e-6))
    if mhd:
        kw.update(induction=True, gamma_m=0.3, eta=0.03, chi=0.4, mu=1.3, B0=(0.01, 0.03, -0.02))
    cfg = orc.Config(nx, ny, nz, **kw)
    S, G = make_pair(orc, cfg, Fext=random_force(nx, ny, nz, 3e-5, seed=5), storage=storage)
    _perturb(S, 17)
    push_oracle_state(S, G)
    fluid = ~S.solid_mask()
    if storage == "bf16":
        # the oracle starts from the state as rounded into BF16
        df0, dg0, _ = gpu_state(G)
        S.f[fluid] = df0[:, fluid].T + W19[None, :] * cfg.rho0
        if mhd:
            S.g[fluid] = dg0[:, fluid].T.reshape(-1, 3, 7) + W7[None, None, :] * np.asarray(cfg.B0)[None, :, None]
    n = 13
    S.run(n)
    G.step(n)
    df, dg, FL = gpu_state(G)
    odf, odg, oFL = oracle_state_dev(S)
    tol = 3e-5 if storage == "f32" else 3e-2
    assert rel_linf(df, odf, fluid) < tol
    if mhd:
        assert rel_linf(dg, odg, fluid) < tol
        assert rel_linf(FL, oFL, fluid) < tol


@pytest.mark.parametrize("nx", [1, 2, 3])
def test_unrolled_adjoint_on_narrow_periodic_ducts(orc, nx):
    from oracle import adjoint as A
    from paper_0809_4730_gb300.inputs import gaussian_force
    cfg = orc.Config(nx, 8, 8, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=0.1, nu=0.05, induction=True,
                     gamma_m=0.1, eta=0.05, chi=0.01, mu=1.0, B0=(0, 2 * 0.05 / 3, 0))
    F = gaussian_force(nx, 8, 8, F0=1e-6, seed=3)
    Faos = np.ascontiguousarray(F.reshape(3, -1).T)
    ref, _ = A.unrolled_gradient(cfg, Faos, A.flow_rate_weights(cfg), 60)
    _, G = make_pair(orc, cfg, F, storage="f32c")
    dQ = G.adjoint_unrolled(60, 11).cpu().double().numpy()
    mask = ~orc.solid_mask(cfg)
    g, r = dQ[:, mask], ref.T[:, mask]
    assert np.abs(g - r).max() / np.abs(r).max() <= 5e-5


# The paired kernel's interior path needs a whole warp (32 pairs) on interior
# rows; with nx = 2 or 4 a warp spans 32 or 16 rows.  Each grid here has at
# least two such warps (counted from the warp-to-row map), and with nx = 2
# both seam corrections apply to the same pair.
PAIR_GEOMETRIES = [
    (2, 57, 6, (0, 1, 1), (0, 1, 1)),
    (2, 45, 6, (0, 0, 0), (0, 0, 0)),
    (4, 30, 5, (0, 1, 0), (0, 1, 1)),
]


@pytest.mark.parametrize("geom", PAIR_GEOMETRIES, ids=[f"{g[0]}x{g[1]}x{g[2]}" for g in PAIR_GEOMETRIES])
@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_paired_step_parity_on_narrow_x(orc, geom, storage):
    from paper_0809_4730_gb300.inputs import random_force
    nx, ny, nz, lo, hi = geom
    cfg = orc.Config(nx, ny, nz, wall_lo=lo, wall_hi=hi, gamma=0.3, nu=0.02, F=(2e-5, -1e-5, 5e-6))
    S, G = make_pair(orc, cfg, Fext=random_force(nx, ny, nz, 3e-5, seed=9), storage=storage, variant=2)
    _perturb(S, 23)
    push_oracle_state(S, G)
    fluid = ~S.solid_mask()
    if storage != "f32":
        df0, _, _ = gpu_state(G)
        S.f[fluid] = df0[:, fluid].T + W19[None, :] * cfg.rho0
    n = 13
    S.run(n)
    G.step(n)
    df, _, _ = gpu_state(G)
    odf, _, _ = oracle_state_dev(S)
    tol = {"f32": 3e-5, "bf16": 3e-2, "f16": 4e-3}[storage]
    assert rel_linf(df, odf, fluid) < tol
