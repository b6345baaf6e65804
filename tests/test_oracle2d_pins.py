"""Pins of the two-dimensional FP64 oracle (D2Q9 GLBE + D2Q5 induction,
arXiv:0809.4730 Secs. 2-4, App. A D2Q9 tables) against what the paper and
the mathematics fix: the velocity-space forms against the moment tables, the
App. A / Sec. 3 numbers as printed (tests/golden/d2q9_tables.txt), closed
forms (Poiseuille, Hartmann, diffusion decay, uniform forcing), conservation,
and a velocity-space SRT-LBE written here in numpy.
"""
import numpy as np
import pytest

from conftest import golden_path

# The test's own statement of the D2Q9 lattice (Eq. velocityd2q9 groups,
# standard weights) in the ordering the oracle and the C-ABI use.
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = np.array([[b for b in range(9) if np.all(E[b] == -E[a])][0] for a in range(9)])
E5 = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1]], dtype=float)


def read_golden():
    eq, src, ps, rates, nm = {}, {}, {}, {}, None
    for line in open(golden_path("d2q9_tables.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "EQ":
            eq[int(t[1])] = np.array(list(map(float, t[2:])))
        elif t[0] == "SRC":
            src[int(t[1])] = np.array(list(map(float, t[2:])))
        elif t[0] == "PS":
            v = list(map(int, t[1:]))
            for k, p in zip(v[0::2], v[1::2]):
                ps[k] = p
        elif t[0] == "RATE":
            rates[int(t[1])] = float(t[2])
        elif t[0] == "NM":
            nm = int(t[1])
    return eq, src, ps, rates, nm


def maxwellian(rho, u, gamma):
    """Preconditioned discrete Maxwellian (Sec. 3.1 form, D2Q9 weights)."""
    eu = E @ u
    return W * rho * (1 + 3 * eu + 4.5 * eu ** 2 / gamma - 1.5 * (u @ u) / gamma)


def source_velocity_space(F, u):
    """S_a = w_a [3 (e_a - u) + 9 (e_a . u) e_a] . F  (Sec. 2)."""
    return W * (3 * ((E - u) @ F) + 9 * (E @ u) * (E @ F))


def source_precond_velocity_space(F, u, gamma):
    """S*_a of the corrected preconditioned source (Sec. 3.1)."""
    return W * (3 * ((E - u / gamma) @ F) / gamma + 9 * (E @ u) * (E @ F) / gamma ** 2)


# ---------------------------------------------------------------------------
# Lattices and the moment matrix
# ---------------------------------------------------------------------------
def test_lattice_ordering_matches(orc2):
    Eo, wo, oppo = orc2.lattice()
    assert np.array_equal(Eo, E.astype(int))
    assert np.allclose(wo, W, rtol=0, atol=1e-16)
    assert np.array_equal(oppo, OPP)
    # second- and fourth-order isotropy of the weights (what the basis needs)
    assert abs(W.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("a,ai,aj->ij", W, E, E), np.eye(2) / 3, atol=1e-16)


def test_moment_matrix_orthogonal_integer(orc2):
    T = orc2.moment_matrix()
    assert np.array_equal(T, np.round(T))
    G = T @ T.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0.0
    assert np.array_equal(T[0], np.ones(9))
    assert np.array_equal(T[3], E[:, 0]) and np.array_equal(T[5], E[:, 1])


@pytest.mark.parametrize("gamma", [1.0, 0.37, 0.05])
def test_equilibrium_moments_are_maxwellian_projection(orc2, gamma):
    T = orc2.moment_matrix()
    rng = np.random.default_rng(11)
    for _ in range(5):
        rho = rng.uniform(0.8, 1.3)
        u = rng.normal(size=2) * 0.05
        m_table = orc2.equilibrium_moments(rho, rho * u, gamma)
        m_proj = T @ maxwellian(rho, u, gamma)
        assert np.allclose(m_table, m_proj, rtol=0, atol=1e-13 * max(1.0, np.abs(m_proj).max()))


def test_equilibrium_moments_match_golden_table(orc2):
    eq, *_ = read_golden()
    rng = np.random.default_rng(3)
    for gamma in (1.0, 0.2):
        rho = 1.1
        j = rng.normal(size=2) * 0.03
        jj = j @ j
        basis = np.array([rho, jj / rho / gamma, j[0], j[1], j[0] ** 2 / rho / gamma, j[1] ** 2 / rho / gamma,
                          j[0] * j[1] / rho / gamma])
        got = orc2.equilibrium_moments(rho, j, gamma)
        want = np.array([eq[k] @ basis for k in range(9)])
        assert np.allclose(got, want, rtol=0, atol=1e-15)


def test_source_moments_are_projection_of_velocity_source(orc2):
    T = orc2.moment_matrix()
    rng = np.random.default_rng(5)
    for _ in range(5):
        F = rng.normal(size=2) * 1e-3
        u = rng.normal(size=2) * 0.05
        assert np.allclose(orc2.source_moments(F, u, 1.0), T @ source_velocity_space(F, u), rtol=0, atol=1e-15)


@pytest.mark.parametrize("gamma", [1.0, 0.5, 0.1, 0.05])
def test_preconditioned_source_inverse_equals_srt_form(orc2, gamma):
    T = orc2.moment_matrix()
    Ti = np.linalg.inv(T)
    rng = np.random.default_rng(7)
    for _ in range(5):
        F = rng.normal(size=2) * 1e-4
        u = rng.normal(size=2) * 0.05
        S_v = Ti @ orc2.source_moments(F, u, gamma)
        assert np.allclose(S_v, source_precond_velocity_space(F, u, gamma), rtol=0, atol=1e-14)


def test_source_table_and_precond_diag_match_golden(orc2):
    _, src, ps, _, _ = read_golden()
    rng = np.random.default_rng(9)
    F = rng.normal(size=2)
    u = rng.normal(size=2)
    basis = np.array([F[0], F[1], F[0] * u[0], F[1] * u[1], F[0] * u[1] + F[1] * u[0]])
    for gamma in (1.0, 0.3):
        got = orc2.source_moments(F, u, gamma)
        want = np.array([src[k] @ basis * gamma ** (-ps[k]) for k in range(9)])
        assert np.allclose(got, want, rtol=1e-14, atol=1e-15)
        assert np.allclose(orc2.source_precond_diag(gamma), [gamma ** (-ps[k]) for k in range(9)], rtol=1e-15)


def test_relaxation_rates_mapping(orc2):
    _, _, _, rates, _ = read_golden()
    s = orc2.relaxation_rates(orc2.Config2(2, 2, gamma=0.2, nu=0.01))
    for k, v in rates.items():
        assert s[k] == v
    snu = 1.0 / (3 * 0.01 / 0.2 + 0.5)
    assert abs(s[7] - snu) < 1e-15 and abs(s[8] - snu) < 1e-15


def test_d2q5_weights_and_equilibrium_moments(orc2):
    """Sec. 4: sum_a g^eq_ja = B_j and sum_a e_ak g^eq_ja = (u_k B_j - B_k u_j)
    chi/gamma_m (the low-Pr_m scaling of Sec. 4.1), from N_m = 3."""
    _, _, _, _, nm = read_golden()
    cfg = orc2.Config2(2, 2, induction=True, gamma_m=0.3, chi=0.4)
    rng = np.random.default_rng(2)
    u, B = rng.normal(size=2) * 0.05, rng.normal(size=2) * 0.02
    geq = orc2.vector_equilibrium(cfg, u, B)
    assert np.allclose(geq.sum(1), B, rtol=0, atol=1e-17)
    first = geq @ E5                                  # [j, k]
    want = (np.outer(B, u) - np.outer(B, u).T) * 0.4 / 0.3
    assert np.allclose(first, want, rtol=0, atol=1e-17)
    # rest weights 1/N_m, 1/(2 N_m)
    geq0 = orc2.vector_equilibrium(cfg, np.zeros(2), np.array([1.0, 0.0]))
    assert np.allclose(geq0[0], [1 / nm] + [1 / (2 * nm)] * 4, atol=1e-16)
    assert abs(orc2.tau_m(orc2.Config2(2, 2, induction=True, gamma_m=0.25, eta=0.05)) - (0.05 / (0.25 / nm) + 0.5)) < 1e-15


# ---------------------------------------------------------------------------
# With every rate 1/tau the MRT-GLBE is the preconditioned SRT-LBE
# (velocity space, written here), also on walls and with a force field.
# ---------------------------------------------------------------------------
def _srt_numpy(f, F, tau, gamma, solid, nsteps):
    f = f.copy()
    for _ in range(nsteps):
        rho = f.sum(0)
        j = np.einsum("a...,ad->d...", f, E) + 0.5 * F / gamma
        u = j / rho
        eu = np.einsum("ad,d...->a...", E, u)
        eF = np.einsum("ad,d...->a...", E, F)
        uu, uF = (u * u).sum(0), (u * F).sum(0)
        feq = W[:, None, None] * rho * (1 + 3 * eu + 4.5 * eu ** 2 / gamma - 1.5 * uu / gamma)
        S = W[:, None, None] * (3 * (eF - uF / gamma) / gamma + 9 * eu * eF / gamma ** 2)
        ft = f - (f - feq) / tau + (1 - 0.5 / tau) * S
        fn = np.empty_like(f)
        for a in range(9):
            sh = (int(E[a, 1]), int(E[a, 0]))
            src = np.roll(ft[a], shift=sh, axis=(0, 1))
            from_solid = np.roll(solid, shift=sh, axis=(0, 1))
            fn[a] = np.where(from_solid, ft[OPP[a]], src)
        f = np.where(solid[None], f, fn)
    return f


@pytest.mark.parametrize("gamma", [1.0, 0.25])
def test_mrt_with_equal_rates_is_preconditioned_srt(orc2, gamma):
    nx, ny = 7, 9
    tau = 0.9
    nu = gamma * (tau - 0.5) / 3.0
    cfg = orc2.Config2(nx, ny, wall_lo=(0, 1), wall_hi=(0, 1), gamma=gamma, nu=nu, s=np.full(9, 1.0 / tau))
    rng = np.random.default_rng(21)
    F = rng.uniform(-1e-4, 1e-4, size=(2, ny, nx))
    S = orc2.Solver2(cfg, Fext=F.reshape(2, -1).T)
    S.f = S.f + rng.uniform(-1e-3, 1e-3, size=S.f.shape) * W
    f0 = S.f.T.reshape(9, ny, nx).copy()
    solid = S.solid_mask().reshape(ny, nx)
    S.run(12)
    got = S.f.T.reshape(9, ny, nx)
    want = _srt_numpy(f0, F, tau, gamma, solid, 12)
    assert np.abs(got[:, ~solid] - want[:, ~solid]).max() < 1e-14


def test_conserved_row_rates_do_not_matter(orc2):
    rng = np.random.default_rng(4)
    F = rng.uniform(-1e-5, 1e-5, size=(6 * 7, 2))
    out = []
    for sval in (1.0, 0.37):
        s = orc2.paper_rates()
        s[[0, 3, 5]] = sval
        cfg = orc2.Config2(6, 7, wall_lo=(0, 1), wall_hi=(0, 1), gamma=0.3, nu=0.02, s=s,
                           induction=True, gamma_m=0.3, eta=0.02, chi=0.5, B0=(0.01, 0.02))
        S = orc2.Solver2(cfg, Fext=F)
        S.f += np.random.default_rng(8).uniform(-1e-3, 1e-3, size=S.f.shape) * W
        S.run(30)
        out.append(S.f.copy())
    assert np.abs(out[0] - out[1]).max() < 1e-15


def test_mass_conservation(orc2):
    rng = np.random.default_rng(12)
    F = rng.uniform(-1e-5, 1e-5, size=(9 * 8, 2))
    cfg = orc2.Config2(9, 8, wall_lo=(1, 1), wall_hi=(0, 1), gamma=0.2, nu=0.02,
                       induction=True, gamma_m=0.2, eta=0.03, chi=0.3, B0=(0.01, 0.03))
    S = orc2.Solver2(cfg, Fext=F)
    S.f += rng.uniform(-1e-3, 1e-3, size=S.f.shape) * W
    fluid = ~S.solid_mask()
    m0 = S.f[fluid].sum()
    S.run(200)
    assert abs(S.f[fluid].sum() - m0) / m0 < 1e-13


@pytest.mark.parametrize("gamma", [1.0, 0.1])
def test_uniform_forcing_momentum_growth(orc2, gamma):
    """Fully periodic, uniform force, rest start: j(t) = (t + 1/2) F/gamma."""
    F = np.array([1e-6, -2e-6])
    S = orc2.Solver2(orc2.Config2(4, 5, gamma=gamma, nu=0.05, F=tuple(F)))
    for t in (0, 7, 40):
        S.run(t - S.t)
        rho, u, _ = S.fields()
        assert np.abs(rho[:, None] * u - (t + 0.5) * F / gamma).max() < 1e-15 * (t + 1)
    S.run(1)
    h = {row["t"]: row for row in S.hist}
    want = 20 * (40 + 0.5) * F / gamma
    assert np.abs(h[40]["mom"] - want).max() <= 1e-12 * np.abs(want).max()


# ---------------------------------------------------------------------------
# Plane Poiseuille (walls y): with Lambda = (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16
# on the energy-flux rows half-way bounce-back gives the parabola up to the
# O(Ma^2) compressibility term; with the paper's rates, second order.
# ---------------------------------------------------------------------------
def _poiseuille(orc2, gamma, nu, ny, F, magic, tol):
    s = orc2.paper_rates()
    if magic:
        snu = 1 / (3 * nu / gamma + 0.5)
        s[[4, 6]] = 1 / (0.5 + (3 / 16) / (1 / snu - 0.5))
    cfg = orc2.Config2(1, ny, wall_lo=(0, 1), wall_hi=(0, 1), gamma=gamma, nu=nu, F=(F, 0), s=s)
    S = orc2.Solver2(cfg)
    S.run(3_000_000, tol=tol)
    _, u, _ = S.fields()
    y = np.arange(ny, dtype=float)
    ana = F * (y - 0.5) * (ny - 1.5 - y) / (2 * nu)
    return S, u[1:-1, 0], ana[1:-1]


@pytest.mark.parametrize("gamma", [0.1, 0.5])
def test_poiseuille_exact_with_magic_rates(orc2, gamma):
    _, u1, a1 = _poiseuille(orc2, gamma, 0.01, 32, 1e-6, True, 1e-13)
    _, u2, a2 = _poiseuille(orc2, gamma, 0.01, 32, 5e-7, True, 1e-13)
    e1 = np.abs(u1 - a1).max() / a1.max()
    e2 = np.abs(u2 - a2).max() / a2.max()
    assert e1 < 2e-6
    assert 3.9 < e1 / e2 < 4.1          # what remains is quadratic in the force


def test_poiseuille_paper_rates_second_order(orc2):
    errs = []
    for ny in (18, 34):
        H = ny - 2
        F = 1e-6 * (16.0 / H) ** 2
        _, u, ana = _poiseuille(orc2, 0.2, 0.02, ny, F, False, 1e-12)
        errs.append(np.abs(u - ana).max() / ana.max())
    assert errs[0] < 5e-3
    assert errs[0] / errs[1] > 3.5


# ---------------------------------------------------------------------------
# Hartmann flow with insulating walls on the 2D lattices (closed form of the
# steady x-momentum and induction equations, Sec. 4.1 scalings):
#   u(y) = F L^2/(rho0 nu Ha tanh Ha) [1 - cosh(Ha y/L)/cosh Ha],
#   b_x(y) = chi B0 A L/(eta Ha cosh Ha) [sinh(Ha y/L) - (y/L) sinh Ha].
# ---------------------------------------------------------------------------
def hartmann2d(orc2, Ha, gamma, ny, F, nu=0.01, eta=0.01, chi=0.01, tol=1e-11):
    L = (ny - 2) / 2
    B0 = Ha * np.sqrt(nu * eta) / L
    cfg = orc2.Config2(1, ny, wall_lo=(0, 1), wall_hi=(0, 1), gamma=gamma, nu=nu, F=(F, 0),
                       induction=True, gamma_m=gamma, eta=eta, chi=chi, mu=1.0, B0=(0, B0))
    S = orc2.Solver2(cfg)
    S.run(5_000_000, tol=tol)
    _, u, B = S.fields()
    y = np.arange(ny) - (ny - 1) / 2
    A = F * L ** 2 / (nu * Ha * np.tanh(Ha))
    ua = A * (1 - np.cosh(Ha * y / L) / np.cosh(Ha))
    ba = chi * B0 * A * L / (eta * Ha * np.cosh(Ha)) * (np.sinh(Ha * y / L) - (y / L) * np.sinh(Ha))
    fl = slice(1, ny - 1)
    eu = np.abs(u[fl, 0] - ua[fl]).max() / ua.max()
    eb = np.abs(B[fl, 0] - ba[fl]).max() / np.abs(ba).max()
    return S, eu, eb, u[fl], B[fl], B0


@pytest.mark.parametrize("Ha,gamma,tol_u", [(5, 0.1, 4e-3), (10, 0.1, 1.2e-2), (5, 1.0, 4e-3)])
def test_hartmann_profile(orc2, Ha, gamma, tol_u):
    S, eu, eb, u, B, B0 = hartmann2d(orc2, Ha, gamma, 64, 1e-6, tol=1e-11 if gamma < 1 else 1e-10)
    assert eu < tol_u
    assert eb < 2.5 * tol_u
    assert u[:, 0].max() < 1e-6 * 31.0 ** 2 / (2 * 0.01)
    assert np.abs(B[:, 1] - B0).max() < 1e-9 * B0 + 1e-15
    assert np.abs(u[:, 1]).max() < 1e-9 * u[:, 0].max()


def test_hartmann_second_order(orc2):
    _, e64, b64, *_ = hartmann2d(orc2, 10, 0.1, 64, 1e-6)
    _, e128, b128, *_ = hartmann2d(orc2, 10, 0.1, 128, 1e-6 * (31.0 / 63.0) ** 2)
    assert e64 / e128 > 3.0
    assert b64 / b128 > 3.0


# ---------------------------------------------------------------------------
# D2Q5 alone (u = 0): a sinusoidal field decays at eta k^2/gamma_m, to O(k^2).
# ---------------------------------------------------------------------------
def _decay_rate(orc2, ny, gamma_m, eta, steps=400, skip=60):
    cfg = orc2.Config2(1, ny, gamma=1.0, nu=0.1, induction=True, gamma_m=gamma_m, eta=eta,
                       chi=1.0, mu=1e30, B0=(0, 0))
    S = orc2.Solver2(cfg)
    y = np.arange(ny)
    b = 1e-4 * np.sin(2 * np.pi * y / ny)
    Wm = np.array([1 / 3] + [1 / 6] * 4)
    S.g[:, 0, :] = b[:, None] * Wm[None, :]
    S.run(skip)
    a1 = np.abs(S.g[:, 0, :].sum(1)).max()
    S.run(steps)
    a2 = np.abs(S.g[:, 0, :].sum(1)).max()
    return np.log(a1 / a2) / steps, eta / gamma_m * (2 * np.pi / ny) ** 2


@pytest.mark.parametrize("gamma_m,eta", [(1.0, 0.05), (0.2, 0.02)])
def test_induction_diffusion_decay(orc2, gamma_m, eta):
    r64, want64 = _decay_rate(orc2, 64, gamma_m, eta)
    r128, want128 = _decay_rate(orc2, 128, gamma_m, eta, steps=1200, skip=120)
    e64 = abs(r64 - want64) / want64
    e128 = abs(r128 - want128) / want128
    assert e64 < 2e-2
    assert e128 < e64 / 3.0 or e128 < 1e-4


def test_current_density_is_curl_of_B(orc2):
    """J_z = (1/(mu chi)) (d_x B_y - d_y B_x) on a smooth field (central
    differences); this fixes the sign reading of J in 2D."""
    n = 128
    chi, mu, eta, gm = 0.5, 2.0, 0.05, 0.5
    cfg = orc2.Config2(n, 1, gamma=1.0, nu=0.1, induction=True, gamma_m=gm, eta=eta, chi=chi, mu=mu, B0=(0, 0))
    S = orc2.Solver2(cfg)
    x = np.arange(n)
    Wm = np.array([1 / 3] + [1 / 6] * 4)
    by = 1e-5 * np.sin(2 * np.pi * x / n)
    bx = 2e-5 * np.cos(2 * np.pi * x / n)     # d_x B_x does not enter J_z
    S.g[:, 0, :] = bx[:, None] * Wm
    S.g[:, 1, :] = by[:, None] * Wm
    S.run(80)
    B = S.g.sum(2)
    Jz = np.array([orc2.current_z(cfg, S.g[k], orc2.vector_equilibrium(cfg, np.zeros(2), B[k])) for k in range(n)])
    want = (np.roll(B[:, 1], -1) - np.roll(B[:, 1], 1)) / 2.0 / (mu * chi)
    assert np.abs(Jz - want).max() / np.abs(want).max() < 5e-3


def test_lorentz_force_is_J_cross_B(orc2):
    """The node's Lorentz force is (-J_z B_y, J_z B_x) with J_z of the
    pre-collision state (Sec. 4, lagged into the next step's force)."""
    cfg = orc2.Config2(2, 2, gamma=0.5, nu=0.05, induction=True, gamma_m=0.5, eta=0.05, chi=0.3, mu=1.0)
    rng = np.random.default_rng(6)
    f = W * (1 + rng.uniform(-1e-3, 1e-3, 9))
    g = np.outer([0.02, -0.01], [1 / 3] + [1 / 6] * 4) + rng.uniform(-1e-4, 1e-4, (2, 5))
    FLprev = np.array([1e-6, -2e-6])
    _, _, mac = orc2.collide_node(cfg, f, g, FLprev)
    B = g.sum(1)
    rho = f.sum()
    u0 = (f @ E + 0.5 * FLprev / 0.5) / rho
    Jz = orc2.current_z(cfg, g, orc2.vector_equilibrium(cfg, u0, B))
    assert np.allclose(mac["FL"], [-Jz * B[1], Jz * B[0]], rtol=1e-14, atol=0)
    assert np.allclose(mac["B"], B, rtol=1e-15, atol=0)


def test_residual_definition(orc2):
    cfg = orc2.Config2(3, 10, wall_lo=(0, 1), wall_hi=(0, 1), gamma=0.5, nu=0.05, F=(1e-5, 0))
    S = orc2.Solver2(cfg)
    fluid = ~S.solid_mask()
    snaps = {}
    for t in (10, 20, 30):
        S.run(t - S.t)
        snaps[t] = S.fields()[1]
    S.run(1)
    h = {row["t"]: row for row in S.hist}
    for t in (20, 30):
        du = snaps[t][fluid] - snaps[t - 10][fluid]
        r = np.sqrt((du ** 2).sum() / (snaps[t][fluid] ** 2).sum())
        assert abs(h[t]["r"] - r) <= 1e-12 * r


def test_equal_preconditioning_of_both_lattices_converges_fastest(orc2):
    """Sec. 5 (Hartmann flow) on the 2D lattices: at gamma = 0.1 the steady
    state comes in the fewest steps at gamma_m = gamma."""
    def steps(gm, Ha=5, ny=34, nu=0.01):
        L = (ny - 2) / 2
        cfg = orc2.Config2(1, ny, wall_lo=(0, 1), wall_hi=(0, 1), gamma=0.1, nu=nu, F=(1e-6, 0),
                           induction=True, gamma_m=gm, eta=nu, chi=0.01, mu=1.0, B0=(0, Ha * nu / L))
        S = orc2.Solver2(cfg)
        S.run(3_000_000, tol=1e-9)
        assert S.hist[-1]["r"] <= 1e-9
        return S.t
    n = {gm: steps(gm) for gm in (1.0, 0.1, 0.05)}
    assert n[0.1] < n[0.05] < n[1.0], n
