"""Pins of the FP64 oracle against what arXiv:0809.4730 and the mathematics fix.

Each test compares the oracle with something other than itself: a second
statement of the paper (velocity-space forms of Sec. 2 and Sec. 3.1 against the
moment tables of App. A), a closed form (Poiseuille, Hartmann, diffusion decay,
uniform forcing), a conservation law, or an independent algorithm (a
velocity-space SRT-LBE written here in numpy, an FD Poisson solve).
"""
import numpy as np
import pytest

from conftest import golden_path

# ---------------------------------------------------------------------------
# The test's own statement of the D3Q19 lattice (Eq. velocityd3q19 groups,
# standard weights) in the ordering the oracle and the C-ABI use.
# ---------------------------------------------------------------------------
E = np.array([[0, 0, 0],
              [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0],
              [1, 0, 1], [-1, 0, 1], [1, 0, -1], [-1, 0, -1],
              [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1]], dtype=float)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
OPP = np.array([[b for b in range(19) if np.all(E[b] == -E[a])][0] for a in range(19)])


def maxwellian(rho, u, gamma):
    """Preconditioned discrete Maxwellian of Sec. 3.1 with the -3/(2 gamma) u.u
    term (the printed -1/(2 gamma) does not reproduce App. A; see DESIGN)."""
    eu = E @ u
    return W * rho * (1 + 3 * eu + 4.5 * eu ** 2 / gamma - 1.5 * (u @ u) / gamma)


def source_velocity_space(F, u):
    """S_a = w_a [3 (e_a - u) + 9 (e_a . u) e_a] . F  (Sec. 2)."""
    return W * (3 * ((E - u) @ F) + 9 * (E @ u) * (E @ F))


def source_precond_velocity_space(F, u, gamma):
    """S*_a of Eq. precondsourcecorrect (Sec. 3.1)."""
    return W * (3 * ((E - u / gamma) @ F) / gamma + 9 * (E @ u) * (E @ F) / gamma ** 2)


def read_golden():
    eq, src, ps, rates = {}, {}, {}, {}
    for line in open(golden_path("d3q19_tables.txt")):
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
    return eq, src, ps, rates


# ---------------------------------------------------------------------------
# P4: the moment matrix
# ---------------------------------------------------------------------------
def test_lattice_ordering_matches(orc):
    Eo, wo, oppo = orc.lattice()
    assert np.array_equal(Eo, E.astype(int))
    assert np.allclose(wo, W, rtol=0, atol=1e-16)
    assert np.array_equal(oppo, OPP)


def test_moment_matrix_orthogonal_integer(orc):
    T = orc.moment_matrix()
    Ti = orc.inverse_moment_matrix()
    assert np.array_equal(T, np.round(T)), "T has integer entries"
    G = T @ T.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0.0, "rows mutually orthogonal"
    assert np.allclose(Ti @ T, np.eye(19), atol=1e-14)
    assert np.allclose(T @ Ti, np.eye(19), atol=1e-14)
    # row 0 is the density, rows 3/5/7 the momentum (Sec. 2, App. A)
    assert np.array_equal(T[0], np.ones(19))
    assert np.array_equal(T[3], E[:, 0]) and np.array_equal(T[5], E[:, 1]) and np.array_equal(T[7], E[:, 2])


# ---------------------------------------------------------------------------
# P1 / P3: equilibrium moments (App. A table, Sec. 3 preconditioned form)
# against the projection of the velocity-space Maxwellian.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gamma", [1.0, 0.37, 0.05])
def test_equilibrium_moments_are_maxwellian_projection(orc, gamma):
    T = orc.moment_matrix()
    rng = np.random.default_rng(11)
    for _ in range(5):
        rho = rng.uniform(0.8, 1.3)
        u = rng.normal(size=3) * 0.05
        m_table = orc.equilibrium_moments(rho, rho * u, gamma)
        m_proj = T @ maxwellian(rho, u, gamma)
        assert np.allclose(m_table, m_proj, rtol=0, atol=1e-13 * max(1.0, np.abs(m_proj).max()))


def test_equilibrium_moments_match_golden_table(orc):
    eq, _, _, _ = read_golden()
    rng = np.random.default_rng(3)
    for gamma in (1.0, 0.2):
        rho = 1.1
        j = rng.normal(size=3) * 0.03
        jj = j @ j
        basis = np.array([rho, jj / rho / gamma, j[0], j[1], j[2],
                          j[0] ** 2 / rho / gamma, j[1] ** 2 / rho / gamma, j[2] ** 2 / rho / gamma,
                          j[0] * j[1] / rho / gamma, j[1] * j[2] / rho / gamma, j[0] * j[2] / rho / gamma])
        got = orc.equilibrium_moments(rho, j, gamma)
        want = np.array([eq[k] @ basis for k in range(19)])
        assert np.allclose(got, want, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# P2 / P3: source moments and their preconditioning
# ---------------------------------------------------------------------------
def test_source_moments_are_projection_of_velocity_source(orc):
    T = orc.moment_matrix()
    rng = np.random.default_rng(5)
    for _ in range(5):
        F = rng.normal(size=3) * 1e-3
        u = rng.normal(size=3) * 0.05
        S_table = orc.source_moments(F, u, 1.0)          # gamma = 1: P_S = I
        S_proj = T @ source_velocity_space(F, u)
        assert np.allclose(S_table, S_proj, rtol=0, atol=1e-15)


@pytest.mark.parametrize("gamma", [1.0, 0.5, 0.1, 0.05])
def test_preconditioned_source_inverse_equals_srt_form(orc, gamma):
    Ti = orc.inverse_moment_matrix()
    rng = np.random.default_rng(7)
    for _ in range(5):
        F = rng.normal(size=3) * 1e-4
        u = rng.normal(size=3) * 0.05
        S_v = Ti @ orc.source_moments(F, u, gamma)
        assert np.allclose(S_v, source_precond_velocity_space(F, u, gamma), rtol=0, atol=1e-14)


def test_source_table_and_precond_diag_match_golden(orc):
    _, src, ps, _ = read_golden()
    rng = np.random.default_rng(9)
    F = rng.normal(size=3)
    u = rng.normal(size=3)
    basis = np.array([F[0], F[1], F[2], F[0] * u[0], F[1] * u[1], F[2] * u[2],
                      F[0] * u[1] + F[1] * u[0], F[1] * u[2] + F[2] * u[1], F[0] * u[2] + F[2] * u[0]])
    for gamma in (1.0, 0.3):
        got = orc.source_moments(F, u, gamma)
        want = np.array([src[k] @ basis * gamma ** (-ps[k]) for k in range(19)])
        assert np.allclose(got, want, rtol=1e-14, atol=1e-15)
        assert np.allclose(orc.source_precond_diag(gamma), [gamma ** (-ps[k]) for k in range(19)], rtol=1e-15)


def test_relaxation_rates_mapping(orc):
    _, _, _, rates = read_golden()
    cfg = orc.Config(2, 2, 2, gamma=0.2, nu=0.01)
    s = orc.relaxation_rates(cfg)
    for k, v in rates.items():
        assert s[k] == v
    snu = 1.0 / (3 * 0.01 / 0.2 + 0.5)
    for k in (9, 11, 13, 14, 15):
        assert abs(s[k] - snu) < 1e-15


# ---------------------------------------------------------------------------
# P5: with every rate equal to 1/tau the MRT-GLBE is the preconditioned
# SRT-LBE of Sec. 3.1 (velocity space), written here independently.
# ---------------------------------------------------------------------------
def _srt_numpy(f, F, tau, gamma, solid, nsteps):
    """Velocity-space preconditioned SRT-LBE, pull streaming with half-way
    bounce-back.  f: [19, nz, ny, nx]; F: [3, nz, ny, nx]."""
    f = f.copy()
    for _ in range(nsteps):
        rho = f.sum(0)
        m = np.einsum("a...,ad->d...", f, E)
        j = m + 0.5 * F / gamma
        u = j / rho
        eu = np.einsum("ad,d...->a...", E, u)
        eF = np.einsum("ad,d...->a...", E, F)
        uu = (u * u).sum(0)
        uF = (u * F).sum(0)
        feq = W[:, None, None, None] * rho * (1 + 3 * eu + 4.5 * eu ** 2 / gamma - 1.5 * uu / gamma)
        S = W[:, None, None, None] * (3 * (eF - uF / gamma) / gamma + 9 * eu * eF / gamma ** 2)
        ft = f - (f - feq) / tau + (1 - 0.5 / tau) * S
        fn = np.empty_like(f)
        for a in range(19):
            sh = (int(E[a, 2]), int(E[a, 1]), int(E[a, 0]))
            src = np.roll(ft[a], shift=sh, axis=(0, 1, 2))
            from_solid = np.roll(solid, shift=sh, axis=(0, 1, 2))
            fn[a] = np.where(from_solid, ft[OPP[a]], src)
        f = np.where(solid[None], f, fn)
    return f


@pytest.mark.parametrize("gamma", [1.0, 0.25])
def test_mrt_with_equal_rates_is_preconditioned_srt(orc, gamma):
    nx, ny, nz = 6, 7, 5
    tau = 0.9
    nu = gamma * (tau - 0.5) / 3.0
    s = np.full(19, 1.0 / tau)
    cfg = orc.Config(nx, ny, nz, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, s=s)
    rng = np.random.default_rng(21)
    F = rng.uniform(-1e-4, 1e-4, size=(3, nz, ny, nx))
    S = orc.Solver(cfg, Fext=F.reshape(3, -1).T)
    S.f = S.f + rng.uniform(-1e-3, 1e-3, size=S.f.shape) * W
    f0 = orc.to_soa(S.f).reshape(19, nz, ny, nx)
    solid = S.solid_mask().reshape(nz, ny, nx)
    S.run(12)
    got = orc.to_soa(S.f).reshape(19, nz, ny, nx)
    want = _srt_numpy(f0, F, tau, gamma, solid, 12)
    fl = ~solid
    assert np.abs(got[:, fl] - want[:, fl]).max() < 1e-14


# ---------------------------------------------------------------------------
# P6: the rates of the conserved rows 0, 3, 5, 7 cannot change the result.
# ---------------------------------------------------------------------------
def test_conserved_row_rates_do_not_matter(orc):
    nx, ny, nz = 5, 6, 4
    rng = np.random.default_rng(4)
    F = rng.uniform(-1e-5, 1e-5, size=(nz * ny * nx, 3))
    out = []
    for sval in (1.0, 0.37):
        s = orc.paper_rates()
        s[[0, 3, 5, 7]] = sval
        cfg = orc.Config(nx, ny, nz, wall_lo=(0, 0, 1), wall_hi=(0, 0, 1), gamma=0.3, nu=0.02, s=s,
                         induction=True, gamma_m=0.3, eta=0.02, chi=0.5, B0=(0.01, 0.02, 0.0))
        S = orc.Solver(cfg, Fext=F)
        S.f += np.random.default_rng(8).uniform(-1e-3, 1e-3, size=S.f.shape) * W
        S.run(30)
        out.append(S.f.copy())
    assert np.abs(out[0] - out[1]).max() < 1e-15


# ---------------------------------------------------------------------------
# P7: mass is conserved exactly (walls, force field, induction coupling).
# ---------------------------------------------------------------------------
def test_mass_conservation(orc):
    nx, ny, nz = 6, 8, 5
    rng = np.random.default_rng(12)
    F = rng.uniform(-1e-5, 1e-5, size=(nz * ny * nx, 3))
    cfg = orc.Config(nx, ny, nz, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=0.2, nu=0.02,
                     induction=True, gamma_m=0.2, eta=0.03, chi=0.3, B0=(0.0, 0.03, 0.01))
    S = orc.Solver(cfg, Fext=F)
    S.f += rng.uniform(-1e-3, 1e-3, size=S.f.shape) * W
    fluid = ~S.solid_mask()
    m0 = S.f[fluid].sum()
    S.run(200)
    m1 = S.f[fluid].sum()
    assert abs(m1 - m0) / m0 < 1e-13


# ---------------------------------------------------------------------------
# The FP64 sums of the residual record (Sec. 5 residual bookkeeping): the mass
# column is the sum of every fluid population at that level (a definition;
# with walls, a force field and induction it also stays at its initial value,
# the scheme conserving mass), and the momentum column is sum rho u.
# ---------------------------------------------------------------------------
def test_history_mass_is_fluid_population_sum(orc):
    nx, ny, nz = 5, 9, 6
    rng = np.random.default_rng(21)
    F = rng.uniform(-1e-5, 1e-5, size=(nz * ny * nx, 3))
    cfg = orc.Config(nx, ny, nz, wall_lo=(0, 1, 1), wall_hi=(0, 1, 0), gamma=0.3, nu=0.03,
                     induction=True, gamma_m=0.3, eta=0.02, chi=0.2, B0=(0.01, 0.02, 0.0))
    S = orc.Solver(cfg, Fext=F)
    S.f += rng.uniform(-2e-3, 2e-3, size=S.f.shape) * W
    fluid = ~S.solid_mask()
    m0 = S.f[fluid].sum()
    sums = {}
    for t in (10, 20, 30):
        S.run(t - S.t)
        sums[t] = S.f[fluid].sum()          # every population of every fluid node at level t
    S.run(1)                                # the record of level 30 is taken when level 30 is collided
    h = {row["t"]: row for row in S.hist}
    for t in (20, 30):
        assert abs(h[t]["mass"] - sums[t]) <= 1e-13 * sums[t]
        assert abs(h[t]["mass"] - m0) <= 1e-13 * m0
    # a solid node's populations never enter the sum
    assert abs(S.f[~fluid].sum()) > 1e-3


@pytest.mark.parametrize("gamma", [1.0, 0.1])
def test_history_momentum_of_uniform_forcing(orc, gamma):
    """P8 through the record: in a fully periodic box under a uniform force
    from rest, sum rho u over the N nodes is N (t + 1/2) F / gamma exactly."""
    F = np.array([2e-6, -1e-6, 5e-7])
    nx, ny, nz = 4, 3, 5
    N = nx * ny * nz
    S = orc.Solver(orc.Config(nx, ny, nz, gamma=gamma, nu=0.05, F=tuple(F)))
    S.run(41)
    h = {row["t"]: row for row in S.hist}
    for t in (20, 30, 40):
        want = N * (t + 0.5) * F / gamma
        assert np.abs(h[t]["mom"] - want).max() <= 1e-12 * np.abs(want).max()
        assert abs(h[t]["mass"] - N * 1.0) <= 1e-13 * N


def test_history_momentum_is_sum_of_j(orc):
    """With walls and a force field the momentum column is the sum over fluid
    nodes of j = sum_a f_a e_a + F/(2 gamma) (Eq. precondhydrofields),
    recomputed here from the populations."""
    nx, ny, nz = 6, 7, 5
    rng = np.random.default_rng(5)
    Fx = rng.uniform(-1e-5, 1e-5, size=(nz * ny * nx, 3))
    gamma = 0.25
    Fu = np.array([1e-6, 0.0, -2e-6])
    S = orc.Solver(orc.Config(nx, ny, nz, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=0.02,
                              F=tuple(Fu)), Fext=Fx)
    S.f += rng.uniform(-1e-3, 1e-3, size=S.f.shape) * W
    fluid = ~S.solid_mask()
    S.run(20)
    j = S.f[fluid] @ E + (Fx[fluid] + Fu) / (2 * gamma)
    S.run(1)
    h = {row["t"]: row for row in S.hist}
    assert np.abs(h[20]["mom"] - j.sum(axis=0)).max() <= 1e-12 * np.abs(j).sum()


# ---------------------------------------------------------------------------
# P8: fully periodic box, uniform force, rest start.  From S*_3 = F/gamma and
# the half-force shift, j(t) = (t + 1/2) F / gamma exactly, state uniform.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gamma", [1.0, 0.1])
def test_uniform_forcing_momentum_growth(orc, gamma):
    F = np.array([1e-6, -2e-6, 3e-6])
    cfg = orc.Config(3, 4, 5, gamma=gamma, nu=0.05, F=tuple(F))
    S = orc.Solver(cfg)
    for t in (0, 7, 40):
        S.run(t - S.t)
        rho, u, _, _ = S.fields()
        j = rho[:, None] * u
        # populations are O(rho): round-off is absolute, about eps per step
        assert np.abs(j - (t + 0.5) * F / gamma).max() < 1e-15 * (t + 1)
        assert np.ptp(S.f, axis=0).max() < 1e-16


# ---------------------------------------------------------------------------
# P9a: plane Poiseuille.  With Lambda = (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16 on
# the third-order rows, half-way bounce-back reproduces the parabola to
# round-off; walls sit half-way between the solid and the first fluid row.
# ---------------------------------------------------------------------------
def _poiseuille(orc, gamma, nu, ny, F, magic, tol):
    s = orc.paper_rates()
    if magic:
        snu = 1 / (3 * nu / gamma + 0.5)
        sq = 1 / (0.5 + (3 / 16) / (1 / snu - 0.5))
        s[[4, 6, 8, 16, 17, 18]] = sq
    cfg = orc.Config(1, ny, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(F, 0, 0), s=s)
    S = orc.Solver(cfg)
    S.run(3_000_000, tol=tol)
    _, u, _, _ = S.fields()
    y = np.arange(ny, dtype=float)
    ana = F * (y - 0.5) * (ny - 1.5 - y) / (2 * nu)
    return S, u[1:-1, 0], ana[1:-1]


@pytest.mark.parametrize("gamma", [0.1, 0.5])
def test_poiseuille_exact_with_magic_rates(orc, gamma):
    # The linear (Stokes) part is exact; what remains is the O(Ma^2)
    # compressibility term, so halving the force quarters the relative error.
    _, u1, a1 = _poiseuille(orc, gamma, 0.01, 32, 1e-6, True, 1e-13)
    _, u2, a2 = _poiseuille(orc, gamma, 0.01, 32, 5e-7, True, 1e-13)
    e1 = np.abs(u1 - a1).max() / a1.max()
    e2 = np.abs(u2 - a2).max() / a2.max()
    assert e1 < 1e-6
    assert 3.5 < e1 / e2 < 4.5


def test_poiseuille_paper_rates_second_order(orc):
    errs = []
    for ny in (18, 34):
        H = ny - 2
        F = 1e-6 * (16.0 / H) ** 2        # hold u_max fixed
        _, u, ana = _poiseuille(orc, 0.2, 0.02, ny, F, False, 1e-12)
        errs.append(np.abs(u - ana).max() / ana.max())
    assert errs[0] < 5e-3
    assert errs[0] / errs[1] > 3.5       # second order in the lattice spacing


def test_paper_poiseuille_case_one(orc):
    """Sec. 5 case 1: L = 32, nu = 0.001, u_max = 0.00051, Re = 32.6."""
    row = [l.split() for l in open(golden_path("poiseuille_cases.txt")) if l.startswith("CASE1")][0]
    L, nu, umax, Re = int(row[1]), float(row[2]), float(row[3]), float(row[4])
    F = 2 * nu * umax / L ** 2               # u_max = F L^2 / (2 rho0 nu)
    # strong preconditioning (the paper runs this case down to gamma = 0.001)
    S, u, ana = _poiseuille(orc, 0.01, nu, 2 * L + 2, F, True, 1e-11)
    assert abs(u.max() - umax) / umax < 2e-3   # centre lies between two nodes
    assert abs(umax * 2 * L / nu - Re) / Re < 2e-3


# ---------------------------------------------------------------------------
# P9b: Hartmann flow with insulating walls.  Derived from the steady x-momentum
# and induction equations of Sec. 4.1 (J = (1/(mu chi)) curl B,
# g^eq with chi/gamma_m): with y measured from the centre and L the half-width,
#   Ha = B0 L / sqrt(mu rho0 nu eta),
#   u(y) = F L^2/(rho0 nu Ha tanh Ha) [1 - cosh(Ha y/L)/cosh Ha],
#   b_x(y) = chi B0 A L/(eta Ha cosh Ha) [sinh(Ha y/L) - (y/L) sinh Ha].
# ---------------------------------------------------------------------------
def hartmann(orc, Ha, gamma, ny, F, nu=0.01, eta=0.01, chi=0.01, tol=1e-11):
    L = (ny - 2) / 2
    B0 = Ha * np.sqrt(nu * eta) / L
    cfg = orc.Config(1, ny, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(F, 0, 0),
                     induction=True, gamma_m=gamma, eta=eta, chi=chi, mu=1.0, B0=(0, B0, 0))
    S = orc.Solver(cfg)
    S.run(5_000_000, tol=tol)
    _, u, B, _ = S.fields()
    y = np.arange(ny) - (ny - 1) / 2
    A = F * L ** 2 / (nu * Ha * np.tanh(Ha))
    ua = A * (1 - np.cosh(Ha * y / L) / np.cosh(Ha))
    ba = chi * B0 * A * L / (eta * Ha * np.cosh(Ha)) * (np.sinh(Ha * y / L) - (y / L) * np.sinh(Ha))
    fl = slice(1, ny - 1)
    eu = np.abs(u[fl, 0] - ua[fl]).max() / ua.max()
    eb = np.abs(B[fl, 0] - ba[fl]).max() / np.abs(ba).max()
    return S, eu, eb, u[fl], B[fl], ua[fl]


@pytest.mark.parametrize("Ha,gamma,tol_u", [(5, 0.1, 4e-3), (10, 0.1, 1.2e-2), (5, 1.0, 4e-3)])
def test_hartmann_profile(orc, Ha, gamma, tol_u):
    S, eu, eb, u, B, ua = hartmann(orc, Ha, gamma, 64, 1e-6, tol=1e-11 if gamma < 1 else 1e-10)
    assert eu < tol_u
    assert eb < 2.5 * tol_u
    # Lorentz drag flattens the profile below the Poiseuille maximum
    L = 31.0
    assert u[:, 0].max() < 1e-6 * L ** 2 / (2 * 0.01)
    # B_y stays the applied field, B_z stays zero
    B0 = Ha * 0.01 / L
    assert np.abs(B[:, 1] - B0).max() < 1e-9 * B0 + 1e-15
    assert np.abs(B[:, 2]).max() < 1e-15


# ---------------------------------------------------------------------------
# Extended induction domain (Sec. 5, MHD cavity): the flow lattice is fluid
# only inside a box, the vector lattice continues outside with u = 0 up to
# the grid's walls, where the induced field is zero.  For the Hartmann layer
# (flow box |y| < L, induction domain |y| < L + e) the exterior is a medium
# of the fluid's magnetic diffusivity at rest: b is linear there, b and b'
# are continuous at the fluid's walls and b(+-(L + e)) = 0, i.e. the Robin
# condition e b'(L) + b(L) = 0.  From the steady x-momentum
# nu u'' + (B0/(mu chi rho0)) b' + F/rho0 = 0 and induction
# eta b'' + chi B0 u' = 0 (Sec. 4.1 scalings):
#   u(y) = K (L/Ha)^2 [1 - cosh(Ha y/L)/cosh Ha],  K = (F + B0 C1/(mu chi))/(rho0 nu),
#   C1 = (chi B0 F/(eta rho0 nu)) (L/Ha)^2 L (1 - tanh(Ha)/Ha) / (e + L tanh(Ha)/Ha);
# e = 0 is the insulating-wall profile above (P9b).
# ---------------------------------------------------------------------------
def hartmann_extended(Ha, L, e, F, nu, eta, chi, B0, y):
    G = (L / Ha) ** 2 * L * (1 - np.tanh(Ha) / Ha)
    C1 = chi * B0 * F / (eta * nu) * G / (e + L * np.tanh(Ha) / Ha)
    K = (F + B0 * C1 / chi) / nu
    return K * (L / Ha) ** 2 * (1 - np.cosh(Ha * y / L) / np.cosh(Ha))


@pytest.mark.parametrize("e", [0, 8, 20])
def test_hartmann_with_extended_induction_domain(orc, e):
    Ha, nu, eta, chi, F = 5.0, 0.01, 0.01, 0.01, 1e-6
    nf = 62                               # fluid rows; half-way walls L = 31 from the centre
    ny = nf + 2 + 2 * e
    L = nf / 2
    B0 = Ha * np.sqrt(nu * eta) / L
    cfg = orc.Config(1, ny, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=0.1, nu=nu, F=(F, 0, 0),
                     induction=True, gamma_m=0.1, eta=eta, chi=chi, mu=1.0, B0=(0, B0, 0),
                     box=((0, 1 + e, 0), (0, ny - 2 - e, 0)))
    S = orc.Solver(cfg)
    S.run(5_000_000, tol=1e-11)
    _, u, B, _ = S.fields()
    y = np.arange(ny) - (ny - 1) / 2
    fl = slice(1 + e, ny - 1 - e)
    ua = hartmann_extended(Ha, L, e, F, nu, eta, chi, B0, y)
    err = np.abs(u[fl, 0] - ua[fl]).max() / ua[fl].max()
    assert err < 4e-3, err
    # outside the box the flow is at rest and the induced field decays to 0 at the grid's walls
    assert np.abs(u[:1 + e]).max() == 0.0
    if e > 0:
        b = B[:, 0]
        assert abs(b[1]) < 0.1 * np.abs(b).max()
    # the conducting exterior changes the flow: e = 0 (insulating) vs e
    if e > 0:
        u0 = hartmann_extended(Ha, L, 0, F, nu, eta, chi, B0, y)
        assert np.abs(ua[fl] - u0[fl]).max() > 20 * 4e-3 * ua[fl].max()


# ---------------------------------------------------------------------------
# Moving wall (Sec. 5, cavity lid; link bounce-back with the wall momentum):
# plane Couette flow between a wall at rest and the lid moving at U is linear,
# u_x(z) = U (z - 1/2)/H with the walls half-way, which half-way bounce-back
# reproduces up to a residue next to the lid of O(U^2/gamma) (the quadratic
# equilibrium terms; 1e-7 U at gamma = 1, 6e-6 U at gamma = 0.1 for
# U = 0.01); preconditioning does not change the steady state otherwise.  A
# wrong sign or factor of the wall term is an O(1) error.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gamma", [1.0, 0.1])
def test_couette_under_the_moving_lid_is_exact(orc, gamma):
    H, U = 24, 0.01
    cfg = orc.Config(1, 1, H + 2, wall_lo=(0, 0, 1), wall_hi=(0, 0, 1), gamma=gamma, nu=0.05, U_lid=(U, 0, 0))
    S = orc.Solver(cfg)
    S.run(5_000_000, tol=1e-13)
    _, u, _, _ = S.fields()
    z = np.arange(H + 2)
    want = U * (z - 0.5) / H
    fl = slice(1, H + 1)
    assert np.abs(u[fl, 0] - want[fl]).max() < 1e-5 * U
    assert np.abs(u[fl, 1:]).max() < 1e-12 * U


def test_hartmann_second_order(orc):
    _, e64, b64, *_ = hartmann(orc, 10, 0.1, 64, 1e-6)
    _, e128, b128, *_ = hartmann(orc, 10, 0.1, 128, 1e-6 * (31.0 / 63.0) ** 2)
    assert e64 / e128 > 3.0
    assert b64 / b128 > 3.0


# ---------------------------------------------------------------------------
# P10: D3Q7 vector lattice alone (u = 0): a sinusoidal field decays at
# eta k^2/gamma_m = theta_m (tau_m - 1/2) k^2 (App. C), to O(k^2) relative.
# ---------------------------------------------------------------------------
def _decay_rate(orc, ny, gamma_m, eta, steps=400, skip=60):
    cfg = orc.Config(1, ny, 1, gamma=1.0, nu=0.1, induction=True, gamma_m=gamma_m, eta=eta,
                     chi=1.0, mu=1e30, B0=(0, 0, 0))
    S = orc.Solver(cfg)
    y = np.arange(ny)
    b = 1e-4 * np.sin(2 * np.pi * y / ny)
    Wm = np.array([0.25] + [0.125] * 6)
    S.g[:, 0, :] = b[:, None] * Wm[None, :]
    S.run(skip)
    a1 = np.abs(S.g[:, 0, :].sum(1)).max()
    S.run(steps)
    a2 = np.abs(S.g[:, 0, :].sum(1)).max()
    return np.log(a1 / a2) / steps, eta / gamma_m * (2 * np.pi / ny) ** 2


@pytest.mark.parametrize("gamma_m,eta", [(1.0, 0.05), (0.2, 0.02)])
def test_induction_diffusion_decay(orc, gamma_m, eta):
    r64, want64 = _decay_rate(orc, 64, gamma_m, eta)
    r128, want128 = _decay_rate(orc, 128, gamma_m, eta, steps=1200, skip=120)
    e64 = abs(r64 - want64) / want64
    e128 = abs(r128 - want128) / want128
    assert e64 < 2e-2
    assert e128 < e64 / 3.0 or e128 < 1e-4


# ---------------------------------------------------------------------------
# P11: the local current density equals (1/(mu chi)) curl B (central
# differences) on a smooth field; this fixes the sign reading of J.
# ---------------------------------------------------------------------------
def test_current_density_is_curl_of_B(orc):
    ny = 128
    chi, mu, eta, gm = 0.5, 2.0, 0.05, 0.5
    cfg = orc.Config(1, ny, 1, gamma=1.0, nu=0.1, induction=True, gamma_m=gm, eta=eta, chi=chi, mu=mu,
                     B0=(0, 0, 0))
    S = orc.Solver(cfg)
    y = np.arange(ny)
    Wm = np.array([0.25] + [0.125] * 6)
    bx = 1e-5 * np.sin(2 * np.pi * y / ny)
    bz = 2e-5 * np.cos(2 * np.pi * y / ny)
    S.g[:, 0, :] = bx[:, None] * Wm
    S.g[:, 2, :] = bz[:, None] * Wm
    S.run(80)
    B = S.g.sum(2)                                      # [N, 3]
    J = np.array([orc.current_density(cfg, S.g[n], orc.vector_equilibrium(cfg, np.zeros(3), B[n]))
                  for n in range(ny)])
    dB = (np.roll(B, -1, axis=0) - np.roll(B, 1, axis=0)) / 2.0     # d/dy
    curl = np.stack([dB[:, 2], np.zeros(ny), -dB[:, 0]], axis=1)    # (dBz/dy, 0, -dBx/dy)
    want = curl / (mu * chi)
    scale = np.abs(want).max()
    assert np.abs(J - want).max() / scale < 5e-3


# ---------------------------------------------------------------------------
# P14: square-duct cross-section with the spatially varying force
# F_x(y, z) against an independent second-order FD Poisson solve
# nu lap(u_x) = -F_x/rho0 with u_x = 0 half-way between solid and fluid.
# ---------------------------------------------------------------------------
def test_duct_against_fd_poisson(orc):
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    from paper_0809_4730_gb300.inputs import duct_force_x
    n = 26
    nu, gamma = 0.05, 0.25
    F = duct_force_x(1, n, n, F0=1e-6)                  # [3, nz, ny, 1]
    s = orc.paper_rates()
    snu = 1 / (3 * nu / gamma + 0.5)
    s[[4, 6, 8, 16, 17, 18]] = 1 / (0.5 + (3 / 16) / (1 / snu - 0.5))
    cfg = orc.Config(1, n, n, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=nu, s=s)
    S = orc.Solver(cfg, Fext=F.reshape(3, -1).T)
    S.run(2_000_000, tol=1e-12)
    _, u, _, _ = S.fields()
    ux = u[:, 0].reshape(n, n)[1:-1, 1:-1]
    m = n - 2
    fx = F[0, 1:-1, 1:-1, 0].reshape(-1)
    # 5-point Laplacian with a ghost value -u at the half-way wall
    main = -4.0 * np.ones((m, m))
    main[0, :] -= 1; main[-1, :] -= 1; main[:, 0] -= 1; main[:, -1] -= 1
    idx = np.arange(m * m).reshape(m, m)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [main.ravel()]
    for dz, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        a = idx[max(dz, 0):m + min(dz, 0), max(dy, 0):m + min(dy, 0)]
        b = idx[max(-dz, 0):m + min(-dz, 0), max(-dy, 0):m + min(-dy, 0)]
        rows.append(a.ravel()); cols.append(b.ravel()); vals.append(np.ones(a.size))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m * m, m * m))
    ufd = spl.spsolve(A * nu, -fx).reshape(m, m)
    assert np.abs(ux - ufd).max() / ufd.max() < 1e-2


# ---------------------------------------------------------------------------
# Residual bookkeeping: r(t) = ||u(t) - u(t-10)|| / ||u(t)|| over fluid nodes.
# ---------------------------------------------------------------------------
def test_residual_definition(orc):
    cfg = orc.Config(3, 10, 4, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=0.5, nu=0.05, F=(1e-5, 0, 0))
    S = orc.Solver(cfg)
    fluid = ~S.solid_mask()
    snaps = {}
    for t in (10, 20, 30):
        S.run(t - S.t)
        snaps[t] = S.fields()[1]
    S.run(1)                   # the residual of level 30 is taken when level 30 is collided
    h = {row["t"]: row for row in S.hist}
    for t in (20, 30):
        du = snaps[t][fluid] - snaps[t - 10][fluid]
        r = np.sqrt((du ** 2).sum() / (snaps[t][fluid] ** 2).sum())
        assert abs(h[t]["r"] - r) <= 1e-12 * r


# ---------------------------------------------------------------------------
# Three statements of the paper's discussion, reproduced by the oracle.
# ---------------------------------------------------------------------------
def test_poiseuille_centre_error_is_linear_in_nu_over_gamma(orc):
    """Sec. 5 (figure of the Poiseuille error): the relative error of the
    centre velocity is linear in nu/gamma.  With the paper's rates only
    s_nu* depends on nu/gamma, and the bounce-back error of the MRT scheme is
    affine in (1/s_nu* - 1/2) = 3 nu/gamma: a straight line to round-off."""
    nu = 0.05
    xs = np.array([0.05, 0.1, 0.2, 0.3, 0.5])
    es = []
    for x in xs:
        _, u, a = _poiseuille(orc, nu / x, nu, 18, 1e-6, False, 1e-12)
        c = len(u) // 2
        es.append((u[c] - a[c]) / a[c])
    es = np.array(es)
    slope, icpt = np.polyfit(xs, es, 1)
    assert np.abs(es - (slope * xs + icpt)).max() < 1e-5 * np.abs(es).max()
    assert abs(slope * (xs[-1] - xs[0])) > 0.1 * np.abs(es).max()     # a real dependence


def test_equal_preconditioning_of_both_lattices_converges_fastest(orc):
    """Sec. 5 (Hartmann flow): with the GLBE at gamma = 0.1, the induction
    lattice reaches the steady state in the fewest steps at gamma_m = gamma;
    gamma_m = 1 is the slowest and gamma_m < gamma is slower again."""
    def steps(gm, Ha=5, ny=34, nu=0.01):
        L = (ny - 2) / 2
        cfg = orc.Config(1, ny, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=0.1, nu=nu, F=(1e-6, 0, 0),
                         induction=True, gamma_m=gm, eta=nu, chi=0.01, mu=1.0, B0=(0, Ha * nu / L, 0))
        S = orc.Solver(cfg)
        S.run(3_000_000, tol=1e-9)
        assert S.hist[-1]["r"] <= 1e-9
        return S.t
    n = {gm: steps(gm) for gm in (1.0, 0.5, 0.1, 0.05)}
    assert n[0.1] < n[0.05] < n[0.5] < n[1.0], n


def test_induction_stays_solenoidal(orc):
    """Sec. 4: the induction remains divergence free when it starts so.  A
    periodic box with a smooth three-component force and an oblique applied
    field: after 2000 steps the central-difference divergence of B is below
    1e-4 of its largest derivative."""
    n = 16
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    k = 2 * np.pi / n
    F = np.stack([np.sin(k * z), np.sin(k * x), np.sin(k * y)], 0) * 2e-5
    cfg = orc.Config(n, n, n, gamma=0.5, nu=0.05, induction=True, gamma_m=0.5, eta=0.05, chi=0.5, mu=1.0,
                     B0=(0.01, 0.03, -0.02))
    S = orc.Solver(cfg, np.ascontiguousarray(F.reshape(3, -1).T))
    S.run(2000)
    _, _, B, _ = S.fields()
    Bf = B.reshape(n, n, n, 3)

    def d(A, ax):
        return (np.roll(A, -1, axis=ax) - np.roll(A, 1, axis=ax)) / 2
    div = d(Bf[..., 0], 2) + d(Bf[..., 1], 1) + d(Bf[..., 2], 0)
    grad = max(np.abs(d(Bf[..., c], ax)).max() for c in range(3) for ax in range(3))
    assert grad > 1e-5
    assert np.abs(div).max() < 1e-4 * grad
