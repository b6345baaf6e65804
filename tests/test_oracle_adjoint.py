"""Pins of the oracle's gradients (oracle/adjoint.py).

The paper has no adjoint; the oracle gradient is the plain definition of the
derivative of the time march (node Jacobians by central differences, the
streaming permutation, and a linear solve or the chain rule).  It is pinned
here against things other than itself:

  - the node Jacobians against what the conservation laws of the update fix
    exactly: mass (sum_a f~_a = sum_a f_a), momentum
    (sum_a e_a f~_a = m + F/gamma with F the total force, Eq.
    precondhydrofields and the conserved rows of Eq. prelax_term), the
    magnetic field (sum_a g~_ja = B_j, Eq. magneticinduction) and the
    velocity u = (m + F/(2 gamma))/rho;
  - the whole gradient against central finite differences of the objective
    through the oracle's own time march (steady solves from rest, or T steps
    from rest), at seeded sample nodes.
"""
import numpy as np
import pytest

E = np.array([[0, 0, 0],
              [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0],
              [1, 0, 1], [-1, 0, 1], [1, 0, -1], [-1, 0, -1],
              [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1]], dtype=float)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
W7 = np.array([0.25] + [0.125] * 6)


def _cfg(orc, nx, n, gamma=0.1, Ha=0.0, nu=0.05):
    L = (n - 2) / 2
    return orc.Config(nx, n, n, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=nu, induction=Ha > 0,
                      gamma_m=gamma, eta=nu, chi=0.01, mu=1.0, B0=(0, Ha * np.sqrt(nu * nu) / L, 0))


def _node_point(rng, induction):
    """A non-equilibrium node state: populations near rest with a flow and a
    field, and forces of the size the workloads use."""
    rho, u = 1.02, np.array([3e-3, -2e-3, 1e-3])
    eu = E @ u
    f = W * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * u @ u) + rng.uniform(-1e-3, 1e-3, 19)
    g = None
    FLp = np.zeros(3)
    if induction:
        B = np.array([1e-3, 3e-2, -2e-3])
        g = (np.outer(B, W7) + rng.uniform(-1e-4, 1e-4, (3, 7))).reshape(21)
        FLp = rng.uniform(-1e-6, 1e-6, 3)
    Fext = np.array([1e-6, 2e-7, -3e-7])
    return f, g, FLp, Fext


@pytest.mark.parametrize("induction", [False, True])
def test_node_jacobian_obeys_the_conservation_laws(orc, induction):
    from oracle import adjoint as A
    rng = np.random.default_rng(5)
    gamma = 0.1
    cfg = orc.Config(4, 4, 4, gamma=gamma, nu=0.05, induction=induction, gamma_m=gamma, eta=0.05, chi=0.01,
                     mu=1.0, B0=(0, 3e-2, 0))
    f, g, FLp, Fext = _node_point(rng, induction)
    J = A.node_jacobian(cfg, f, g, FLp, Fext, A.fd_steps(cfg, 1e-6))
    ft, _, mac = orc.collide_node(cfg, f, g, FLp, Fext)
    rho, u = mac["rho"], mac["u"]
    ncol = 46
    # d(input)/d(input_k) for the f, g, F_L, F_ext blocks
    eye = np.eye(ncol)
    dFL = J[40:43] if induction else np.zeros((3, ncol))
    dF = dFL + eye[43:46]                      # total force F = F_ext + F_L
    dm = np.zeros((3, ncol))
    dm[:, :19] = E.T                           # m = sum_a f_a e_a
    drho = np.zeros(ncol)
    drho[:19] = 1.0
    cols = np.r_[0:19, 43:46] if not induction else np.arange(ncol)
    # rounding of the central differences: ~1e-16 |f~| / h, h = 1e-6 for the
    # populations and 1e-9 for the forces
    tol = np.where(np.arange(ncol) >= 40, 2e-7, 2e-9)[cols]

    def close(a, b):
        assert np.all(np.abs(a - b) <= tol), np.max(np.abs(a - b) / tol)
    # mass
    close(J[:19].sum(0)[cols], drho[cols])
    # momentum: sum_a e_a f~_a = m + F/gamma
    for c in range(3):
        close((E.T @ J[:19])[c, cols], (dm + dF / gamma)[c, cols])
    # velocity: u = (m + F/(2 gamma)) / rho
    du = (dm + dF / (2 * gamma) - np.outer(u, drho)) / rho
    for c in range(3):
        close(J[43 + c, cols], du[c, cols])
    if induction:
        # B_j = sum_a g~_ja = sum_a g_ja
        dB = np.zeros((3, ncol))
        for j in range(3):
            dB[j, 19 + 7 * j:26 + 7 * j] = 1.0
        for j in range(3):
            close(J[19:40].reshape(3, 7, ncol).sum(1)[j], dB[j])
        # the new Lorentz force sees F_ext and the previous one only through their
        # sum in u0 = (m + (F_ext + F_L^prev)/(2 gamma))/rho (coupling reading)
        np.testing.assert_allclose(J[40:43, 43:46], J[40:43, 40:43], rtol=1e-6, atol=1e-12)


@pytest.mark.slow
def test_steady_gradient_matches_finite_differences(orc):
    """12^3 duct with the induction lattice (Ha = 5, gamma = 0.1): the oracle's
    steady gradient against central differences of two steady solves."""
    from oracle import adjoint as A
    from paper_0809_4730_gb300 import inputs
    n = 12
    cfg = _cfg(orc, n, n, Ha=5.0)
    F = np.ascontiguousarray(inputs.gaussian_force(n, n, n, seed=1).reshape(3, -1).T)
    w = A.flow_rate_weights(cfg)
    tol = 5e-12
    dQ, _, _ = A.steady_gradient(cfg, F, w, tol=tol)
    scale = np.abs(dQ).max()
    fluid = np.flatnonzero(~orc.solid_mask(cfg))
    rng = np.random.default_rng(3)
    for k in range(3):
        node = int(rng.choice(fluid))
        fd = A.fd_steady(cfg, F, w, node, k, 1e-8, tol=tol)
        assert abs(fd - dQ[node, k]) <= 1e-6 * scale, (node, k, fd, dQ[node, k])


@pytest.mark.parametrize("Ha", [0.0, 2.0])
def test_unrolled_gradient_matches_finite_differences(orc, Ha):
    """6 x 8 x 8 duct, 60 steps from rest: the chain rule against central
    differences of the 60-step march."""
    from oracle import adjoint as A
    from paper_0809_4730_gb300 import inputs
    cfg = _cfg(orc, 6, 8, Ha=Ha)
    F = np.ascontiguousarray(inputs.gaussian_force(6, 8, 8, seed=1).reshape(3, -1).T)
    w = A.flow_rate_weights(cfg)
    dQ, _ = A.unrolled_gradient(cfg, F, w, 60)
    scale = np.abs(dQ).max()
    fluid = np.flatnonzero(~orc.solid_mask(cfg))
    rng = np.random.default_rng(3)
    for k in range(4):
        node = int(rng.choice(fluid))
        c = k % 3
        fd = A.fd_unrolled(cfg, F, w, 60, node, c, 1e-8)
        assert abs(fd - dQ[node, c]) <= 1e-7 * scale, (node, c, fd, dQ[node, c])


def test_gradient_vanishes_on_solid_nodes(orc):
    from oracle import adjoint as A
    from paper_0809_4730_gb300 import inputs
    cfg = _cfg(orc, 6, 8, Ha=0.0)
    F = np.ascontiguousarray(inputs.gaussian_force(6, 8, 8, seed=1).reshape(3, -1).T)
    dQ, _ = A.unrolled_gradient(cfg, F, A.flow_rate_weights(cfg), 20)
    assert np.all(dQ[orc.solid_mask(cfg)] == 0.0)
