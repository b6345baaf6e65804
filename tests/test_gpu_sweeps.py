"""Stability and preconditioning sweeps through the batch engine (Sec. 5:
Poiseuille stability, Hartmann gamma_m studies): many small problems in one
persistent launch.

- gamma_min(u_max): the smallest gamma of a sweep at which a plane channel
  stays finite rises with the Mach number (the paper's Poiseuille
  discussion: the minimum stable gamma is higher at higher Ma).
- At gamma = 0.05 the Hartmann channel converges in the fewest steps at
  gamma_m = gamma, gamma_m = 1 is the slowest (the paper's Hartmann
  gamma_m studies); a converged domain's level matches the FP64 oracle's.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_minimum_stable_gamma_rises_with_mach():
    import bench
    gammas = (1.0, 0.2, 0.1, 0.05, 0.02, 0.01, 0.005)
    smap = bench.stability_map(nus=(0.005, 0.02), umaxs=(0.005, 0.02, 0.04), gammas=gammas, max_steps=40_000)
    assert smap["domains"] == 2 * 3 * len(gammas)
    for nu in (0.005, 0.02):
        cells = sorted((c for c in smap["map"] if c["nu"] == nu), key=lambda c: c["u_max"])
        gmin = [c["gamma_min"] for c in cells]
        assert all(g is not None for g in gmin)
        assert all(a <= b for a, b in zip(gmin, gmin[1:])), (nu, gmin)
        assert gmin[-1] > gmin[0], (nu, gmin)
        assert all(c["status"]["1.0"] != "diverged" for c in cells)


def test_equal_preconditioning_is_fastest_and_matches_the_oracle(orc):
    import bench
    res = bench.gamma_m_sweep(Ha=10.0, gammas=(0.05,), gms=(1.0, 0.2, 0.05, 0.02), max_steps=400_000)
    row = res["gamma_0.05"]
    assert row["fastest"] == "gamma_m_0.05", row
    assert row["gamma_m_1.0"] > 3 * row["gamma_m_0.05"]
    # the batch's converged level against the oracle's march of the same channel
    nu = 0.01
    H = 62
    B0 = 10.0 * nu / (H / 2)
    cfg = orc.Config(1, H + 2, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=0.05, nu=nu, F=(1e-6, 0, 0),
                     induction=True, gamma_m=0.05, eta=nu, chi=0.01, mu=1.0, B0=(0, B0, 0))
    S = orc.Solver(cfg)
    S.run(1_000_000, tol=1e-8)
    assert abs(row["gamma_m_0.05"] - S.t) <= 20, (row["gamma_m_0.05"], S.t)
