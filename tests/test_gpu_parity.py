"""Parity of the CUDA library (through its C-ABI) with the FP64 oracle.

Tolerances (FP32 arithmetic and storage, unit round-off u = 2^-24 = 6e-8):
one step applies about 30 floating-point operations to every population, so a
step adds at most ~30 u relative to the largest deviation D; over n steps the
error stays below n * 30 u * D.  For the 23-step cases that is 4e-5 D; the
tests use 3e-5 D, the tail of a random walk being far below the worst case.
BF16 storage rounds every population once per step to 8 bits (u = 2^-9 =
2e-3 relative); FP16 with the default scale 4096 to 11 bits (u = 2.4e-4).
At steady state the bar is the stated one: velocity L-infinity relative
error <= 1e-5 against the converged FP64 oracle.
"""
import numpy as np
import pytest

from gpu_common import (W19, W7, gpu_fields, gpu_state, make_pair, oracle_state_dev, push_oracle_state,
                        rel_linf, require_cuda)

pytestmark = pytest.mark.gpu


def _cfg(orc, mhd, gamma=0.3, nx=37, ny=11, nz=9, **kw):
    base = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 0), gamma=gamma, nu=0.02, F=(2e-5, -1e-5, 5e-6))
    if mhd:
        base.update(induction=True, gamma_m=gamma, eta=0.03, chi=0.4, mu=1.3, B0=(0.01, 0.03, -0.02))
    base.update(kw)
    return orc.Config(nx, ny, nz, **base)


def _perturb(S, seed, scale=2e-3):
    from paper_0809_4730_gb300.inputs import perturbation
    cfg = S.cfg
    p = perturbation(19, cfg.nx, cfg.ny, cfg.nz, scale, seed).reshape(19, -1).T
    S.f += p * W19[None, :]
    if cfg.induction:
        q = perturbation(21, cfg.nx, cfg.ny, cfg.nz, scale * 0.05, seed + 1).reshape(21, -1).T
        S.g += q.reshape(cfg.N, 3, 7) * W7[None, None, :]
        S.FL[:] = perturbation(3, cfg.nx, cfg.ny, cfg.nz, 1e-6, seed + 2).reshape(3, -1).T


def _check_record_sums(info, row, S, fluid, tol):
    """The GPU record's mass and momentum against the oracle record of the
    same level.  Both are compared through their deviations: sum drho =
    mass - rho0 N_fluid, which the scheme conserves, and sum j.  The bound is
    tol times (fluid nodes x the largest population deviation, resp. the
    largest |j|): far below rho0 N_fluid, so a dropped, doubled or
    solid-node term is seen."""
    cfg = S.cfg
    nf = int(fluid.sum())
    odf, _, _ = oracle_state_dev(S)
    D = np.abs(odf[:, fluid]).max()
    rho, u, _, _ = S.fields()
    jmax = np.abs(rho[fluid, None] * u[fluid]).max()
    m0 = cfg.rho0 * nf
    assert abs((info.mass - m0) - (row["mass"] - m0)) <= tol * nf * D, (info.mass - m0, row["mass"] - m0)
    assert np.abs(np.array(info.momentum[:]) - row["mom"]).max() <= tol * nf * jmax, \
        (info.momentum[:], row["mom"])


@pytest.mark.parametrize("mhd", [False, True])
def test_state_roundtrip_is_exact(orc, mhd):
    cfg = _cfg(orc, mhd)
    S, G = make_pair(orc, cfg)
    _perturb(S, 5)
    push_oracle_state(S, G)
    df, dg, FL = gpu_state(G)
    odf, odg, oFL = oracle_state_dev(S)
    fluid = ~S.solid_mask()
    assert np.array_equal(df[:, fluid], odf[:, fluid].astype(np.float32).astype(np.float64))
    if mhd:
        assert np.array_equal(dg[:, fluid], odg[:, fluid].astype(np.float32).astype(np.float64))
        assert np.array_equal(FL[:, fluid], oFL[:, fluid].astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("storage", ["f32", "f32c"])
@pytest.mark.parametrize("mhd", [False, True])
@pytest.mark.parametrize("gamma", [1.0, 0.3])
def test_step_parity_f32(orc, mhd, gamma, storage):
    from paper_0809_4730_gb300.inputs import random_force
    cfg = _cfg(orc, mhd, gamma=gamma)
    Fext = random_force(cfg.nx, cfg.ny, cfg.nz, 3e-5, seed=7)
    S, G = make_pair(orc, cfg, Fext=Fext, storage=storage)
    _perturb(S, 11)
    push_oracle_state(S, G)
    fluid = ~S.solid_mask()
    nsteps = 23
    S.run(nsteps)
    G.step(nsteps)
    df, dg, FL = gpu_state(G)
    odf, odg, oFL = oracle_state_dev(S)
    assert rel_linf(df, odf, fluid) < 3e-5
    if mhd:
        assert rel_linf(dg, odg, fluid) < 3e-5
        assert rel_linf(FL, oFL, fluid) < 3e-5
    rho, u, B = gpu_fields(G)
    orho, ou, oB, _ = S.fields()
    # rho leaves the library as an FP32 number near rho0: its own rounding
    # (2^-24 rho0) adds to the deviation error
    drho = np.abs(orho[fluid] - cfg.rho0).max()
    assert np.abs(rho[fluid] - orho[fluid]).max() <= 3e-5 * drho + 2 ** -24 * cfg.rho0
    assert rel_linf(u, ou.T, fluid) < 3e-5
    if mhd:
        assert rel_linf(B, oB.T, fluid) < 3e-5
    # residual of level 20 (evaluated inside the step that collided it)
    info = G.residual()
    h = {row["t"]: row for row in S.hist}
    assert info.t == 20
    assert abs(info.r - h[20]["r"]) <= 1e-3 * h[20]["r"]
    _check_record_sums(info, h[20], S, fluid, 3e-5)


# A stochastically rounded value is off by less than one unit in the last
# place (round-to-nearest: half a unit), zero on average: twice the bound.
@pytest.mark.parametrize("storage,tol", [("bf16", 3e-2), ("f16", 4e-3), ("bf16sr", 6e-2), ("f16sr", 8e-3)])
def test_step_parity_reduced_storage(orc, storage, tol):
    from paper_0809_4730_gb300.inputs import random_force
    cfg = _cfg(orc, True, gamma=0.5)
    Fext = random_force(cfg.nx, cfg.ny, cfg.nz, 3e-5, seed=3)
    S, G = make_pair(orc, cfg, Fext=Fext, storage=storage)
    _perturb(S, 13)
    push_oracle_state(S, G)
    # the oracle starts from the state as rounded into the reduced storage
    df0, dg0, FL0 = gpu_state(G)
    fluid = ~S.solid_mask()
    odf, odg, _ = oracle_state_dev(S)
    assert rel_linf(df0, odf, fluid) < (8e-3 if storage.startswith("bf16") else 1e-3)
    S.f[fluid] = (df0[:, fluid].T + W19[None, :] * cfg.rho0)
    B0 = np.asarray(cfg.B0)
    S.g[fluid] = dg0[:, fluid].T.reshape(-1, 3, 7) + W7[None, None, :] * B0[None, :, None]
    n = 15
    S.run(n)
    G.step(n)
    df, dg, _ = gpu_state(G)
    odf, odg, _ = oracle_state_dev(S)
    assert rel_linf(df, odf, fluid) < tol
    assert rel_linf(dg, odg, fluid) < tol
    _, u, _ = gpu_fields(G)
    _, ou, _, _ = S.fields()
    assert rel_linf(u, ou.T, fluid) < tol


def test_nonfinite_state_is_reported_as_divergence(orc):
    from paper_0809_4730_gb300.glbe import GLBE_ERR_DIVERGED, GlbeError
    torch = require_cuda()
    cfg = _cfg(orc, False)
    S, G = make_pair(orc, cfg)
    push_oracle_state(S, G)
    df, _, _ = G.get_state()
    fluid_idx = int(np.flatnonzero(~S.solid_mask())[5])
    df[3, fluid_idx] = float("nan")
    G.set_state(df, t=0)
    G.step(21)
    with pytest.raises(GlbeError) as ei:
        G.residual()
    assert ei.value.status == GLBE_ERR_DIVERGED


# The paired kernel (two x-adjacent nodes per thread, packed FP32x2): even nx,
# x periodic.  nx = 2 and 6 make rows shorter than a warp, so every
# row-start, row-end and warp-edge case of its lane shuffles occurs; nx = 38
# leaves a partial last warp.
# nx = 38 and 66: warps straddle rows; nx = 64: a warp of 32 pairs covers one
# row.  The flow forms with 16-bit or F32 storage gather the warps that lie
# wholly on interior rows at fixed offsets (every nx here but 2 and 6 has such
# warps), the rest through the row geometry.
@pytest.mark.parametrize("nx", [2, 6, 38, 64, 66])
@pytest.mark.parametrize("storage,tol", [("f32", 3e-5), ("bf16", 3e-2), ("f32c", 3e-5), ("bf16sr", 6e-2),
                                         ("f16sr", 8e-3)])
@pytest.mark.parametrize("mhd", [False, True])
def test_step_parity_paired_kernel(orc, nx, storage, tol, mhd):
    from paper_0809_4730_gb300.inputs import random_force
    cfg = _cfg(orc, mhd, gamma=0.4, nx=nx, ny=9, nz=7)
    Fext = random_force(cfg.nx, cfg.ny, cfg.nz, 3e-5, seed=nx)
    S, G = make_pair(orc, cfg, Fext=Fext, storage=storage, variant=2)
    _perturb(S, 17 + nx)
    push_oracle_state(S, G)
    fluid = ~S.solid_mask()
    if storage != "f32":
        # start the oracle from the state as rounded into the storage
        df0, dg0, FL0 = gpu_state(G)
        S.f[fluid] = (df0[:, fluid].T + W19[None, :] * cfg.rho0)
        if mhd:
            B0 = np.asarray(cfg.B0)
            S.g[fluid] = dg0[:, fluid].T.reshape(-1, 3, 7) + W7[None, None, :] * B0[None, :, None]
    n = 13
    S.run(n)
    G.step(n)
    df, dg, FL = gpu_state(G)
    odf, odg, oFL = oracle_state_dev(S)
    assert rel_linf(df, odf, fluid) < tol
    if mhd:
        assert rel_linf(dg, odg, fluid) < tol
        assert rel_linf(FL, oFL, fluid) < max(tol, 3e-5)
    # the residual of level 10 was formed by the paired kernel's block sums
    info = G.residual()
    h = {row["t"]: row for row in S.hist}
    assert info.t == 10
    assert abs(info.r - h[10]["r"]) <= max(1e-3, 30 * tol) * h[10]["r"]
    _check_record_sums(info, h[10], S, fluid, max(tol, 3e-5))


# The TMA-staged tile kernel (variant 3): x periodic, nx a multiple of 128.
# It gathers the same values as the one-node kernel and runs the same node
# update, so the states must agree bit for bit; ny = 9 with walls on both
# y planes and nz = 7 with one z wall leave fluid rows next to walls, rows
# that wrap around z, and the x seam at x = 0 / nx - 1.
@pytest.mark.parametrize("nx", [128, 256])
@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("mhd", [False, True])
def test_tile_kernel_matches_one_node_kernel_bitwise(orc, nx, storage, mhd):
    from paper_0809_4730_gb300.inputs import random_force
    cfg = _cfg(orc, mhd, gamma=0.4, nx=nx, ny=9, nz=7)
    Fext = random_force(cfg.nx, cfg.ny, cfg.nz, 3e-5, seed=nx)
    S, G1 = make_pair(orc, cfg, Fext=Fext, storage=storage, variant=1)
    _, G3 = make_pair(orc, cfg, Fext=Fext, storage=storage, variant=3)
    _perturb(S, 23 + nx)
    push_oracle_state(S, G1)
    push_oracle_state(S, G3)
    G1.step(21)
    G3.step(21)
    for a, b in zip(gpu_state(G1), gpu_state(G3)):
        if a is not None:
            assert np.array_equal(a, b)
    r1, r3 = G1.residual(), G3.residual()
    assert r1.t == r3.t == 20
    assert abs(r1.r - r3.r) <= 1e-5 * r1.r        # block sums in another order
    assert abs(r1.mass - r3.mass) <= 1e-9 * r1.mass


# The coupled compensated steps (and the FP32 and BF16 residual steps) run in two passes per thread
# (induction, then flow with this step's Lorentz force) under the automatic choice on
# grids of more than two resident waves of the one-pass kernel (152 SMs x one
# or two blocks of 256 nodes): the one-pass arithmetic in the same
# order, bit for bit, with walls on y and z (general-path nodes), the x seam,
# a force field and two residual levels.
@pytest.mark.parametrize("storage", ["f32c", "f32", "bf16"])
@pytest.mark.parametrize("nx,walls", [(37, ((0, 1, 1), (0, 1, 0))), (64, ((1, 1, 0), (0, 1, 1)))])
def test_coupled_two_pass_matches_one_pass_bitwise(orc, nx, walls, storage):
    from paper_0809_4730_gb300.inputs import random_force
    cfg = _cfg(orc, True, gamma=0.3, nx=nx, ny=64, nz=80, wall_lo=walls[0], wall_hi=walls[1])
    assert cfg.nx * cfg.ny * cfg.nz > 4 * 152 * 256
    Fext = random_force(cfg.nx, cfg.ny, cfg.nz, 3e-5, seed=31)
    S, G0 = make_pair(orc, cfg, Fext=Fext, storage=storage, variant=0)
    _, G1 = make_pair(orc, cfg, Fext=Fext, storage=storage, variant=1)
    _perturb(S, 29)
    push_oracle_state(S, G0)
    push_oracle_state(S, G1)
    G0.step(23)
    G1.step(23)
    for a, b in zip(gpu_state(G0), gpu_state(G1)):
        assert np.array_equal(a, b)
    r0, r1 = G0.residual(), G1.residual()
    assert r0.t == r1.t == 20
    assert (r0.num, r0.den, r0.mass) == (r1.num, r1.den, r1.mass)
    for a, b in zip(gpu_fields(G0), gpu_fields(G1)):
        assert np.array_equal(a, b)


# Variant 4: the tile kernel with two x-adjacent nodes per consumer thread
# runs the paired kernel's packed FP32x2 update on the same gathered values:
# bit-identical to variant 2.
@pytest.mark.parametrize("nx", [128, 256])
@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("mhd", [False, True])
def test_paired_tile_kernel_matches_paired_kernel_bitwise(orc, nx, storage, mhd):
    from paper_0809_4730_gb300.inputs import random_force
    cfg = _cfg(orc, mhd, gamma=0.4, nx=nx, ny=9, nz=7)
    Fext = random_force(cfg.nx, cfg.ny, cfg.nz, 3e-5, seed=nx + 1)
    S, G2 = make_pair(orc, cfg, Fext=Fext, storage=storage, variant=2)
    _, G4 = make_pair(orc, cfg, Fext=Fext, storage=storage, variant=4)
    _perturb(S, 29 + nx)
    push_oracle_state(S, G2)
    push_oracle_state(S, G4)
    G2.step(21)
    G4.step(21)
    for a, b in zip(gpu_state(G2), gpu_state(G4)):
        if a is not None:
            assert np.array_equal(a, b)
    r2, r4 = G2.residual(), G4.residual()
    assert r2.t == r4.t == 20
    assert abs(r2.r - r4.r) <= 1e-5 * r2.r


_CAPTURE_FIRST = """
import sys
import numpy as np
import torch
from paper_0809_4730_gb300.glbe import Solver
kw = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 0), gamma=0.5, nu=0.1, F=(2e-5, -1e-5, 5e-6), storage="f32")
out = []
for v in (1, int(sys.argv[1])):
    G = Solver(128, 9, 7, variant=v, **kw)
    st, n, r = G.solve(1e-6, 200_000)    # the first launches of this process are captured in a graph
    df, _, _ = G.get_state()
    G.sync()
    out.append((st, n, df.cpu().numpy()))
assert out[0][0] == out[1][0] == 0, out
assert abs(out[0][1] - out[1][1]) <= 10
if sys.argv[1] == "3":
    assert out[0][1] == out[1][1] and np.array_equal(out[0][2], out[1][2])
print("ok")
"""


@pytest.mark.parametrize("variant", [3, 4])
def test_tile_kernel_first_used_inside_a_captured_solve(variant):
    """In a fresh process whose first steps are the CUDA-graph chunks of
    glbe_solve, the tile kernel's one-time set-up runs during stream capture;
    the solve must match the one-node kernel's."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CAPTURE_FIRST, str(variant)], cwd=root, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("storage,tol", [("f32", 3e-5), ("bf16", 3e-2)])
@pytest.mark.parametrize("mhd", [False, True])
@pytest.mark.parametrize("variant", [3, 4])
def test_step_parity_tile_kernel(orc, storage, tol, mhd, variant):
    from paper_0809_4730_gb300.inputs import random_force
    cfg = _cfg(orc, mhd, gamma=0.4, nx=128, ny=9, nz=7)
    Fext = random_force(cfg.nx, cfg.ny, cfg.nz, 3e-5, seed=5)
    S, G = make_pair(orc, cfg, Fext=Fext, storage=storage, variant=variant)
    _perturb(S, 41)
    push_oracle_state(S, G)
    fluid = ~S.solid_mask()
    if storage != "f32":
        df0, dg0, FL0 = gpu_state(G)
        S.f[fluid] = (df0[:, fluid].T + W19[None, :] * cfg.rho0)
        if mhd:
            B0 = np.asarray(cfg.B0)
            S.g[fluid] = dg0[:, fluid].T.reshape(-1, 3, 7) + W7[None, None, :] * B0[None, :, None]
    n = 13
    S.run(n)
    G.step(n)
    df, dg, FL = gpu_state(G)
    odf, odg, oFL = oracle_state_dev(S)
    assert rel_linf(df, odf, fluid) < tol
    if mhd:
        assert rel_linf(dg, odg, fluid) < tol
        assert rel_linf(FL, oFL, fluid) < max(tol, 3e-5)
    G.sync()


# ---------------------------------------------------------------------------
# Steady state: plane channel 4x32x4 (walls at y = 0, 31), F_x = 1e-6,
# tau = 0.8 on the stress moments, gamma = 0.1.  The oracle runs the x/z-
# invariant column 1x32x1 (identical problem) to r <= 1e-10.
# ---------------------------------------------------------------------------
def _channel(orc, gamma, nu, ny=32):
    return orc.Config(1, ny, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0))


def test_steady_channel_parity(orc):
    from paper_0809_4730_gb300.glbe import Solver
    gamma = 0.1
    nu = gamma * (0.8 - 0.5) / 3.0
    S = orc.Solver(_channel(orc, gamma, nu))
    S.run(2_000_000, tol=1e-10)
    _, ou, _, _ = S.fields()
    G = Solver(4, 32, 4, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0))
    st, steps, r = G.solve(1e-9, 400_000)
    _, u, _ = gpu_fields(G)
    ux = u[0].reshape(4, 32, 4)
    col = ux[:, :, :].transpose(1, 0, 2).reshape(32, -1)           # [y, (z,x)]
    want = ou[:, 0]
    err = np.abs(col - want[:, None]).max() / np.abs(want).max()
    assert err <= 1e-5, f"velocity L-inf relative error {err:.3e} (GPU r = {r:.2e} after {steps} steps)"


def test_preconditioning_cuts_steps(orc):
    """Steps to r <= 1e-8 on the channel: gamma = 0.1 at least 5x fewer than
    gamma = 1 at the same physical viscosity.  The GPU residual history
    (every 10 levels) follows the oracle's: r(t) agrees within 5 % while
    r > 1e-7 (the crossing step of 1e-8 itself is sensitive: near it r falls
    by only ~0.1 % per evaluation at gamma = 1)."""
    from paper_0809_4730_gb300.glbe import Solver
    nu = 0.1 * 0.3 / 3.0
    counts = {}
    for gamma in (1.0, 0.1):
        S = orc.Solver(_channel(orc, gamma, nu))
        S.run(2_000_000, tol=1e-8)
        G = Solver(1, 32, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0),
                   storage="f32c")
        G.step(4000)
        hist = {h["t"]: h["r"] for h in G.history()}
        for row in S.hist:
            if row["t"] in hist and row["r"] > 1e-7:
                assert abs(hist[row["t"]] - row["r"]) <= 0.05 * row["r"], (gamma, row["t"], hist[row["t"]], row["r"])
        st, steps, r = G.solve(1e-8, 2_000_000)
        assert st == 0 and r <= 1e-8
        assert abs(steps - S.t) <= 0.15 * S.t, (gamma, steps, S.t)
        counts[gamma] = steps
    assert counts[1.0] >= 5 * counts[0.1]


# ---------------------------------------------------------------------------
# Steady Hartmann duct 64x64x8 (walls at y = 0, 63), B0 along y, Pr_m = 0.01,
# nu = eta = 0.01, gamma = gamma_m = 0.1; oracle on the 1x64x1 column.
# ---------------------------------------------------------------------------
def _hartmann_oracle(orc, Ha, gamma, nu=0.01, eta=0.01, chi=0.01):
    L = 31.0
    B0 = Ha * np.sqrt(nu * eta) / L
    cfg = orc.Config(1, 64, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0),
                     induction=True, gamma_m=gamma, eta=eta, chi=chi, mu=1.0, B0=(0, B0, 0))
    S = orc.Solver(cfg)
    S.run(3_000_000, tol=1e-10)
    return cfg, S


@pytest.mark.parametrize("storage", ["f32", "f32c"])
@pytest.mark.parametrize("Ha,gamma", [(5, 0.1), (10, 0.1), (20, 0.1), (10, 1.0)])
def test_steady_hartmann_parity(orc, Ha, gamma, storage):
    from paper_0809_4730_gb300.glbe import Solver
    nu = eta = 0.01
    chi = 0.01
    L = 31.0
    B0 = Ha * np.sqrt(nu * eta) / L
    cfg = orc.Config(1, 64, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0),
                     induction=True, gamma_m=gamma, eta=eta, chi=chi, mu=1.0, B0=(0, B0, 0))
    S = orc.Solver(cfg)
    S.run(3_000_000, tol=1e-10)
    _, ou, oB, _ = S.fields()
    G = Solver(64, 64, 8, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0), induction=1,
               gamma_m=gamma, eta=eta, chi=chi, mu=1.0, B0=(0, B0, 0), storage=storage)
    st, steps, r = G.solve(1e-9, 1_000_000)
    _, u, B = gpu_fields(G)
    ux = u[0].reshape(8, 64, 64).transpose(1, 0, 2).reshape(64, -1)
    bx = B[0].reshape(8, 64, 64).transpose(1, 0, 2).reshape(64, -1)
    fl = slice(1, 63)
    eu = np.abs(ux[fl] - ou[fl, 0][:, None]).max() / np.abs(ou[fl, 0]).max()
    eb = np.abs(bx[fl] - oB[fl, 0][:, None]).max() / np.abs(oB[fl, 0]).max()
    # F32C meets the FP32 bar of 1e-5; plain FP32 storage keeps the
    # stagnation error of its slowest mode: measured 1-2e-5 at gamma = 0.1
    # (bound 3e-5) and 6.3e-5 at Ha = 10, gamma = 1 (bound 1e-4)
    bar = 1e-5 if storage == "f32c" else (1e-4 if gamma == 1.0 else 3e-5)
    assert eu <= bar, f"u error {eu:.3e} (GPU r = {r:.2e}, {steps} steps)"
    assert eb <= 1e-4, f"b error {eb:.3e}"


@pytest.mark.parametrize("storage,bound", [("f32c", 1e-5), ("f32", 3e-5), ("f16", 5e-2), ("bf16", 5e-1),
                                           ("f16sr", 5e-2), ("bf16sr", 5e-1)])
def test_steady_accuracy_per_storage(orc, storage, bound):
    """Steady Hartmann (Ha = 10, gamma = 0.1) after a fixed 40000 steps: the
    error of each storage form against the converged FP64 oracle.  The
    16-bit forms stall where the needed corrections fall below half a unit in
    the last place of the stored deviation (error ~ ulp / decay rate of the
    slowest mode); FP32 with exact-split moments keeps that floor near 1e-5,
    the compensated form removes it."""
    from paper_0809_4730_gb300.glbe import Solver
    cfg, S = _hartmann_oracle(orc, 10, 0.1)
    _, ou, _, _ = S.fields()
    G = Solver(64, 64, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=cfg.gamma, nu=cfg.nu, F=cfg.F, induction=1,
               gamma_m=cfg.gamma_m, eta=cfg.eta, chi=cfg.chi, mu=1.0, B0=cfg.B0, storage=storage)
    G.step(40_000)
    info = G.residual()
    _, u, _ = gpu_fields(G)
    ux = u[0].reshape(64, 64)
    fl = slice(1, 63)
    err = np.abs(ux[fl] - ou[fl, 0][:, None]).max() / np.abs(ou[fl, 0]).max()
    print(f"steady accuracy {storage}: rel L-inf error {err:.3e}, residual r({info.t}) = {info.r:.3e}")
    assert err <= bound


# ---------------------------------------------------------------------------
# The 64^3 copy of the square duct (walls y, z; x periodic; F_x(y, z) of the
# duct workload, F0 = 1e-6, nu = 0.5).  Its steady state is x-invariant, so
# the oracle solves the 1 x 64 x 64 column, the same discrete problem, to
# r <= 1e-11.
# ---------------------------------------------------------------------------
def _duct64_oracle(orc, gamma, n=64):
    from paper_0809_4730_gb300.inputs import duct_force_x
    F = duct_force_x(1, n, n)[0].reshape(-1)
    Fext = np.zeros((n * n, 3))
    Fext[:, 0] = F
    S = orc.Solver(orc.Config(1, n, n, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=0.5), Fext=Fext)
    S.run(2_000_000, tol=1e-11)
    _, ou, _, _ = S.fields()
    return S, ou[:, 0].reshape(n, n)


def _duct64_gpu(storage, gamma, n=64):
    from paper_0809_4730_gb300.glbe import Solver
    from paper_0809_4730_gb300.inputs import duct_force_x
    torch = require_cuda()
    G = Solver(n, n, n, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=0.5, force_field=1, storage=storage)
    G.set_force(torch.tensor(duct_force_x(n, n, n)[0].reshape(1, -1), dtype=torch.float32, device="cuda"))
    return G


def _duct64_error(G, col, n=64):
    _, u, _ = gpu_fields(G)
    ux = u[0].reshape(n, n, n)[1:-1, 1:-1, :]
    c = col[1:-1, 1:-1]
    return np.abs(ux - c[:, :, None]).max() / np.abs(c).max()


# Bounds about twice the errors measured on a GB300 after 6000-12000 steps
# (F32C 1.5e-7, F32 1.6e-7, F16 2.9e-4, BF16 1.8e-3, F16_SR 5-7e-4, BF16_SR
# 4.4-4.9e-3).  The 16-bit forms leave the error of their stored precision:
# round-to-nearest stagnates (error ~ ulp / decay rate), stochastic rounding
# leaves zero-mean noise of about one ulp.
@pytest.mark.parametrize("storage,bound", [("f32c", 1e-6), ("f32", 1e-6), ("f16", 1e-3), ("bf16", 5e-3),
                                           ("f16sr", 2e-3), ("bf16sr", 1.2e-2)])
def test_duct64_steady_accuracy_per_storage(orc, storage, bound):
    _, col = _duct64_oracle(orc, 0.1)
    G = _duct64_gpu(storage, 0.1)
    G.step(6000)
    err = _duct64_error(G, col)
    info = G.residual()
    print(f"64^3 duct steady error {storage}: {err:.3e}, r({info.t}) = {info.r:.3e}")
    assert err <= bound
    G.close()


@pytest.mark.parametrize("gamma", [1.0, 0.1])
def test_duct64_compensated_march_reaches_1e8(orc, gamma):
    """The compensated form solves the 64^3 duct to r <= 1e-8 (the residual
    keeps u as a double-float pair, so FP32 rounding of u does not floor it)
    within 25 % of the oracle's step count, at the FP32 bar of 1e-5."""
    S, col = _duct64_oracle(orc, gamma)
    t8 = min(h["t"] for h in S.hist if h["r"] <= 1e-8)
    G = _duct64_gpu("f32c", gamma)
    st, steps, r = G.solve(1e-8, 200_000)
    assert st == 0 and r <= 1e-8, (st, steps, r)
    assert abs(steps - t8) <= 0.25 * t8, (steps, t8)
    assert _duct64_error(G, col) <= 1e-5
    G.close()


# ---------------------------------------------------------------------------
# Full size, bench launch configuration: the 256x256x512 square duct with
# F_x(y, z).  One step from a seeded random state; sampled nodes are checked
# against the oracle's single-node collision and the streaming map.
# ---------------------------------------------------------------------------
E19 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                [1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0], [1, 0, 1], [-1, 0, 1], [1, 0, -1], [-1, 0, -1],
                [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1]])
OPP19 = np.array([0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15])


@pytest.mark.parametrize("storage,tol", [("f32", 2e-6), ("bf16", 2e-3)])
def test_full_size_duct_sampled(orc, storage, tol):
    from paper_0809_4730_gb300.glbe import Solver
    from paper_0809_4730_gb300.inputs import duct_force_x
    torch = require_cuda()
    nx, ny, nz = 512, 256, 256
    N = nx * ny * nz
    gamma, nu = 0.1, 0.5
    G = Solver(nx, ny, nz, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=nu, force_field=1,
               storage=storage)
    F = duct_force_x(nx, ny, nz)[0].reshape(1, -1)
    G.set_force(torch.tensor(F, dtype=torch.float32, device="cuda"))
    gen = torch.Generator(device="cuda").manual_seed(0)
    df0 = (torch.rand(19, N, device="cuda", generator=gen) - 0.5) * 2e-3 * torch.tensor(
        W19, dtype=torch.float32, device="cuda")[:, None]
    G.set_state(df0, t=1)
    pre, _, _ = G.get_state()
    G.step(1)
    post, _, _ = G.get_state()
    G.sync()
    rng = np.random.default_rng(1)
    xs, ys, zs = rng.integers(0, nx, 64), rng.integers(1, ny - 1, 64), rng.integers(1, nz - 1, 64)
    # include wall-adjacent and periodic-edge nodes
    xs[:4], ys[:4], zs[:4] = [0, nx - 1, 5, 9], [1, ny - 2, 1, ny - 2], [1, nz - 2, nz - 2, 1]
    cfg = orc.Config(nx, ny, nz, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=nu)
    idx = torch.tensor((zs * ny + ys) * nx + xs, device="cuda")
    pre_s = pre[:, idx].double().cpu().numpy()
    worst = 0.0
    for k in range(len(xs)):
        x, y, z = int(xs[k]), int(ys[k]), int(zs[k])
        n = (z * ny + y) * nx + x
        f = pre_s[:, k] + W19
        ft, _, _ = orc.collide_node(cfg, f, Fext=np.array([F[0, n], 0.0, 0.0]))
        dft = ft - W19
        for a in range(19):
            xt, yt, zt = (x + E19[a, 0]) % nx, y + E19[a, 1], z + E19[a, 2]
            if yt in (0, ny - 1) or zt in (0, nz - 1):
                got = post[OPP19[a], n]
            else:
                got = post[a, (zt * ny + yt) * nx + xt]
            worst = max(worst, abs(float(got) - dft[a]) / 1e-3)
    assert worst < tol
