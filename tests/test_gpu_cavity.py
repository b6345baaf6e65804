"""The cavity kernel (a fluid box and / or a moving lid; Sec. 5, 3D
lid-driven cavity and its MHD case on an extended magnetic domain) through
the C-ABI, against the FP64 oracle and closed forms.

- Per step: a lid-driven cavity (walls on all faces, lid moving along x),
  with and without the induction lattice on an extended domain around the
  flow box, marched 23 steps from rest, compared node by node with the
  oracle's march (u on the fluid nodes, B on every node off the walls).
- Couette under the lid: the linear profile (oracle pin).
- Hartmann flow with an extended induction domain: the closed form with a
  conducting exterior (oracle pin) and the converged oracle.
- The steady cavity flow is mirror-symmetric about the mid-plane normal to
  the lid's spanwise direction: u_y odd, u_x and u_z even.
"""
import numpy as np
import pytest

from gpu_common import gpu_fields, require_cuda

pytestmark = pytest.mark.gpu


def _cfgs(orc, mhd, storage, n=14, e=3, U=0.02, gamma=0.3):
    kw = dict(wall_lo=(1, 1, 1), wall_hi=(1, 1, 1), gamma=gamma, nu=0.05, U_lid=(U, 0.0, 0.0))
    box = ((1 + e, 1 + e, 1 + e), (n - 2 - e, n - 2 - e, n - 2 - e)) if mhd else None
    if mhd:
        kw.update(induction=True, gamma_m=gamma, eta=0.05, chi=0.3, mu=1.0, B0=(0.0, 0.02, 0.0))
    cfg = orc.Config(n, n, n, box=box, **kw)
    gkw = dict(kw, storage=storage, box=box)
    gkw["induction"] = int(mhd)
    return cfg, gkw


@pytest.mark.parametrize("storage,tol", [("f32", 3e-5), ("f32c", 3e-5), ("bf16", 3e-2)])
@pytest.mark.parametrize("mhd", [False, True])
def test_cavity_step_parity(orc, storage, tol, mhd):
    from paper_0809_4730_gb300.glbe import Solver
    require_cuda()
    cfg, gkw = _cfgs(orc, mhd, storage)
    S = orc.Solver(cfg)
    G = Solver(cfg.nx, cfg.ny, cfg.nz, **gkw)
    S.run(23)
    G.step(23)
    _, u, B = gpu_fields(G)
    _, ou, oB, _ = S.fields()
    fluid = ~S.solid_mask()
    ref = ou.T[:, fluid]
    assert np.abs(u[:, fluid] - ref).max() <= tol * np.abs(ref).max()
    assert np.abs(u[:, ~fluid]).max() == 0.0
    if mhd:
        walls = orc.Config(cfg.nx, cfg.ny, cfg.nz, wall_lo=cfg.wall_lo, wall_hi=cfg.wall_hi)
        live = ~orc.solid_mask(walls)
        B0 = np.asarray(cfg.B0)[:, None]
        got = B[:, live] - B0
        want = oB.T[:, live] - B0
        assert np.abs(got - want).max() <= tol * np.abs(want).max() + 2 ** -24 * 0.02
    info = G.residual()
    h = {row["t"]: row for row in S.hist}
    assert info.t == 20 and abs(info.r - h[20]["r"]) <= max(1e-3, 30 * tol) * h[20]["r"]
    G.close()


@pytest.mark.parametrize("storage", ["f32", "f32c"])
def test_coupled_cavity_two_pass_matches_one_pass_bitwise(orc, storage):
    """The coupled cavity step of the FP32 forms in two passes per thread
    (the automatic choice) against the one-pass kernel (variant 1): the same
    fields and residual sums bit for bit after 23 steps (the lid, the box
    faces, the extended magnetic domain and two residual levels)."""
    from paper_0809_4730_gb300.glbe import Solver
    require_cuda()
    cfg, gkw = _cfgs(orc, True, storage)
    G0 = Solver(cfg.nx, cfg.ny, cfg.nz, variant=0, **gkw)
    G1 = Solver(cfg.nx, cfg.ny, cfg.nz, variant=1, **gkw)
    G0.step(23)
    G1.step(23)
    for a, b in zip(gpu_fields(G0), gpu_fields(G1)):
        assert np.array_equal(a, b)
    r0, r1 = G0.residual(), G1.residual()
    assert (r0.t, r0.num, r0.den, r0.mass) == (r1.t, r1.num, r1.den, r1.mass)
    G0.close()
    G1.close()


def test_couette_under_the_lid():
    from paper_0809_4730_gb300.glbe import Solver
    require_cuda()
    H, U = 24, 0.01
    G = Solver(1, 1, H + 2, wall_lo=(0, 0, 1), wall_hi=(0, 0, 1), gamma=0.1, nu=0.05, U_lid=(U, 0, 0),
               storage="f32c")
    st, steps, r = G.solve(1e-8, 2_000_000)
    assert st == 0, (steps, r)
    _, u, _ = gpu_fields(G)
    z = np.arange(H + 2)
    want = U * (z - 0.5) / H
    assert np.abs(u[0, 1:H + 1] - want[1:H + 1]).max() < 1e-5 * U
    G.close()


@pytest.mark.parametrize("e", [0, 8])
def test_hartmann_with_extended_induction_domain(orc, e):
    from paper_0809_4730_gb300.glbe import Solver
    from test_oracle_pins import hartmann_extended
    require_cuda()
    Ha, nu, eta, chi, F = 5.0, 0.01, 0.01, 0.01, 1e-6
    nf = 62
    ny = nf + 2 + 2 * e
    L = nf / 2
    B0 = Ha * np.sqrt(nu * eta) / L
    box = ((0, 1 + e, 0), (0, ny - 2 - e, 0))
    kw = dict(wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=0.1, nu=nu, F=(F, 0, 0), gamma_m=0.1, eta=eta, chi=chi,
              mu=1.0, B0=(0, B0, 0))
    S = orc.Solver(orc.Config(1, ny, 1, induction=True, box=box, **kw))
    S.run(5_000_000, tol=1e-11)
    _, ou, _, _ = S.fields()
    G = Solver(1, ny, 1, induction=1, box=box, storage="f32c", **kw)
    st, steps, r = G.solve(1e-9, 5_000_000)
    assert st == 0
    _, u, _ = gpu_fields(G)
    fl = slice(1 + e, ny - 1 - e)
    y = np.arange(ny) - (ny - 1) / 2
    ua = hartmann_extended(Ha, L, e, F, nu, eta, chi, B0, y)
    assert np.abs(u[0, fl] - ou[fl, 0]).max() <= 1e-5 * ou[fl, 0].max()
    assert np.abs(u[0, fl] - ua[fl]).max() <= 4e-3 * ua[fl].max()
    G.close()


def test_steady_cavity_is_mirror_symmetric():
    """Lid along x, walls on every face: the flow is symmetric about the
    mid-plane y = (ny - 1)/2 (u_y odd, u_x and u_z even).  The march is
    taken to r <= 1e-6: at the edges of the lid, where the velocity jumps,
    preconditioning raises the density deviations to ~1e-2 and the FP32
    collide arithmetic keeps r near 1-2e-7 (the FP64 oracle converges)."""
    from paper_0809_4730_gb300.glbe import Solver
    require_cuda()
    n = 18
    G = Solver(n, n, n, wall_lo=(1, 1, 1), wall_hi=(1, 1, 1), gamma=0.2, nu=0.05, U_lid=(0.05, 0, 0),
               storage="f32c")
    st, steps, r = G.solve(1e-6, 2_000_000)
    assert st == 0, (steps, r)
    G.step(2000)
    _, u, _ = gpu_fields(G)
    u = u.reshape(3, n, n, n)                 # [c][z][y][x]
    m = u[:, :, ::-1, :]
    s = np.abs(u).max()
    assert np.abs(u[0] - m[0]).max() <= 1e-5 * s
    assert np.abs(u[2] - m[2]).max() <= 1e-5 * s
    assert np.abs(u[1] + m[1]).max() <= 1e-5 * s
    # the lid drives a primary vortex: u_x > 0 under the lid, < 0 near the bottom
    assert u[0, n - 2, n // 2, n // 2] > 0 and u[0, 2, n // 2, n // 2] < 0
    G.close()
