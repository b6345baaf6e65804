"""FP64 oracle gradients of a velocity objective with respect to the
body-force field.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

The paper (arXiv:0809.4730) has no adjoint; what is computed here is the
plain definition of the derivative of its time march:

  objective   Q = sum_x w(x) . u(x), with u the velocity of Eq.
              precondhydrofields (j / rho with the half force) at the state
              the objective is taken on; the flow-rate objective is
              w = (1/L_x, 0, 0) on every fluid node, L_x the number of fluid
              planes along x, so Q = (1/L_x) sum_fluid u_x.

  state       s = per node (f[19], g[21], F_L[3]) before collision: the
              quantities one time step reads (Secs. 2-4; F_L is the Lorentz
              force of the previous step, see the oracle's coupling reading).

  step        s_{t+1} = P Y(s_t, F): Y is the node update (collision, new
              Lorentz force), P the streaming of Eqs. pstreaming/mstreaming
              with bounce-back (f) and anti-bounce-back (g), identity on F_L.

  steady      s* = P Y(s*, F) together with the mass of the initial state:
              the march conserves m.s = sum over fluid nodes of sum_a f_a, so
              I - P Y_s is singular along the mass mode and the fixed point
              is unique only with that constraint.  The implicit function
              theorem on the bordered system gives
                dQ/dF = U_F^t w + Y_F^t P^t lam,
                (I - P Y_s)^t lam + beta m = U_s^t w,   m.lam = 0,
              solved by GMRES (scipy.sparse.linalg) to a 1e-12 relative
              residual.  (The forcing adds no mass, m.P Y_F = 0, so the mass
              multiplier beta does not enter dQ/dF.)

  unrolled    s_0 = rest state, Q on s_T; the chain rule backwards:
              lam_T = U_s(T)^t w, and for t = T-1 .. 0:
              v = P^t lam_{t+1},  dQ/dF += Y_F(t)^t v,  lam_t = Y_s(t)^t v;
              plus U_F(T)^t w.

The node Jacobians Y_s, Y_F, U_s, U_F come from ``orc_state_jacobians``
(central differences of the oracle's node update in FP64).  Everything else
is sparse linear algebra on those blocks and the streaming permutation P,
built here from the push rule of the oracle's step (a population leaving x
along e_a lands on x + e_a, or, when that node is solid, returns to x in the
opposite slot; for g with the sign flipped).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import Config, Solver, _p, lattice, lib, solid_mask

NJ = 46            # node map inputs / outputs: f 19, g 21, F_L 3, F_ext or u 3
U_ROWS = slice(43, 46)
F_COLS = slice(43, 46)

# D3Q7 ordering of the oracle (0 rest, +x, -x, +y, -y, +z, -z)
E7 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
OPP7 = np.array([0, 2, 1, 4, 3, 6, 5])


def state_dim(cfg: Config) -> int:
    return 43 if cfg.induction else 19


def fd_steps(cfg: Config, F_scale: float) -> np.ndarray:
    """Central-difference steps per input column: populations O(0.1) take
    1e-6; g (O(W B0)) and the forces (O(F_scale)) a step relative to their
    own scale, so that rounding (~1e-16 |y| / h) stays near 1e-10 of the
    derivative."""
    h = np.empty(NJ)
    h[:19] = 1e-6 * cfg.rho0
    Bs = max(float(np.max(np.abs(cfg.B0))), 1e-3)
    h[19:40] = 1e-4 * Bs
    h[40:46] = 1e-3 * max(F_scale, 1e-9)
    return h


def state_jacobians(cfg: Config, f: np.ndarray, g: np.ndarray, FL: np.ndarray, Fext: np.ndarray | None,
                    h: np.ndarray) -> np.ndarray:
    """[N, 46, 46] node Jacobians of a state (oracle AoS arrays)."""
    p = cfg.params()
    J = np.zeros((cfg.N, NJ, NJ))
    Fe = None if Fext is None else np.ascontiguousarray(Fext, dtype=np.float64).reshape(cfg.N, 3)
    lib().orc_state_jacobians(C.byref(p), _p(np.ascontiguousarray(f)),
                              _p(np.ascontiguousarray(g)) if cfg.induction else None,
                              _p(np.ascontiguousarray(FL)), _p(Fe), _p(np.ascontiguousarray(h)), _p(J))
    return J


def node_jacobian(cfg: Config, f, g, FLprev, Fext, h) -> np.ndarray:
    """[46, 46] Jacobian of one node's update (total external force Fext)."""
    p = cfg.params()
    J = np.zeros(NJ * NJ)
    f = np.ascontiguousarray(f, dtype=np.float64)
    gg = np.ascontiguousarray(np.zeros(21) if g is None else g, dtype=np.float64).reshape(21)
    fl = np.ascontiguousarray(np.zeros(3) if FLprev is None else FLprev, dtype=np.float64)
    fe = np.ascontiguousarray(Fext, dtype=np.float64)
    lib().orc_node_jacobian(C.byref(p), _p(f), _p(gg), _p(fl), _p(fe), _p(np.ascontiguousarray(h)), _p(J))
    return J.reshape(NJ, NJ)


def flow_rate_weights(cfg: Config) -> np.ndarray:
    """w[N, 3] of Q = (1/L_x) sum_fluid u_x."""
    Lx = cfg.nx - int(cfg.wall_lo[0]) - int(cfg.wall_hi[0])
    w = np.zeros((cfg.N, 3))
    w[~solid_mask(cfg), 0] = 1.0 / Lx
    return w


def streaming_matrix(cfg: Config) -> sp.csr_matrix:
    """P: post-collision values (per node: f~ 19, g~ 21, F_L 3) -> the next
    step's pre-collision state, for fluid target nodes (rows of solid nodes
    are empty)."""
    nd = state_dim(cfg)
    E, _, opp = lattice()
    nx, ny, nz = cfg.nx, cfg.ny, cfg.nz
    solid = solid_mask(cfg)
    rows, cols, vals = [], [], []
    for n in range(cfg.N):
        if solid[n]:
            continue
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        # push from node n along a: to n + e_a, or bounced back into n
        for a in range(19):
            xt, yt, zt = (x + E[a, 0]) % nx, (y + E[a, 1]) % ny, (z + E[a, 2]) % nz
            m = (zt * ny + yt) * nx + xt
            if solid[m]:
                rows.append(n * nd + opp[a]); cols.append(n * nd + a); vals.append(1.0)
            else:
                rows.append(m * nd + a); cols.append(n * nd + a); vals.append(1.0)
        if cfg.induction:
            for a in range(7):
                xt, yt, zt = (x + E7[a, 0]) % nx, (y + E7[a, 1]) % ny, (z + E7[a, 2]) % nz
                m = (zt * ny + yt) * nx + xt
                for j in range(3):
                    src = n * nd + 19 + j * 7 + a
                    if solid[m]:
                        rows.append(n * nd + 19 + j * 7 + OPP7[a]); cols.append(src); vals.append(-1.0)
                    else:
                        rows.append(m * nd + 19 + j * 7 + a); cols.append(src); vals.append(1.0)
            for c in range(3):
                rows.append(n * nd + 40 + c); cols.append(n * nd + 40 + c); vals.append(1.0)
    M = cfg.N * nd
    return sp.csr_matrix((vals, (rows, cols)), shape=(M, M))


def _block_diag(blocks: np.ndarray) -> sp.bsr_matrix:
    N, r, c = blocks.shape
    return sp.bsr_matrix((blocks, np.arange(N), np.arange(N + 1)), shape=(N * r, N * c))


def _split(cfg: Config, J: np.ndarray):
    nd = state_dim(cfg)
    Ys = J[:, :nd, :nd]
    YF = J[:, :nd, F_COLS]
    Us = J[:, U_ROWS, :nd]
    UF = J[:, U_ROWS, F_COLS]
    return Ys, YF, Us, UF


def _oracle_state(S: Solver):
    g = S.g.reshape(S.cfg.N, 21) if S.cfg.induction else np.zeros((S.cfg.N, 21))
    return S.f.copy(), g.copy(), S.FL.copy()


def objective(S: Solver, w: np.ndarray) -> float:
    """Q = sum w . u of the solver's current state."""
    _, u, _, _ = S.fields()
    return float(np.sum(w * u))


def steady_state(cfg: Config, Fext: np.ndarray | None, tol: float, max_steps: int) -> Solver:
    S = Solver(cfg, Fext)
    S.run(max_steps, tol)
    if not S.hist or not (S.hist[-1]["r"] <= tol):
        raise RuntimeError(f"oracle steady solve did not reach r <= {tol} in {max_steps} steps")
    return S


def steady_gradient(cfg: Config, Fext: np.ndarray | None, w: np.ndarray, tol: float = 1e-11,
                    max_steps: int = 2_000_000, F_scale: float = 1e-6, S: Solver | None = None):
    """dQ/dF [N, 3] at the steady state (returns (dQdF, lam, solver))."""
    if S is None:
        S = steady_state(cfg, Fext, tol, max_steps)
    f, g, FL = _oracle_state(S)
    J = state_jacobians(cfg, f, g, FL, S.Fext, fd_steps(cfg, F_scale))
    Ys, YF, Us, UF = _split(cfg, J)
    P = streaming_matrix(cfg)
    A = (P @ _block_diag(Ys)).tocsr()
    b = np.einsum("nc,nck->nk", w, Us).reshape(-1)
    nd = state_dim(cfg)
    m = np.zeros((cfg.N, nd))
    m[~solid_mask(cfg), :19] = 1.0
    m = m.reshape(-1)
    K = (sp.identity(A.shape[0], format="csr") - A).T
    Kb = sp.bmat([[K, sp.csr_matrix(m[:, None])], [sp.csr_matrix(m[None, :]), None]]).tocsr()
    rhs = np.concatenate([b, [0.0]])
    x, info = spla.gmres(Kb, rhs, rtol=1e-12, atol=0.0, restart=300, maxiter=100)
    res = np.linalg.norm(Kb @ x - rhs) / np.linalg.norm(rhs)
    if info != 0 or not res <= 1e-10:
        raise RuntimeError(f"adjoint GMRES did not converge (info {info}, relative residual {res:.2e})")
    lam = x[:-1]
    v = (P.T @ lam).reshape(cfg.N, -1)
    dQdF = np.einsum("nc,ncd->nd", w, UF) + np.einsum("ni,nid->nd", v, YF)
    return dQdF, lam, S


def unrolled_gradient(cfg: Config, Fext: np.ndarray | None, w: np.ndarray, nsteps: int,
                      F_scale: float = 1e-6):
    """dQ/dF [N, 3] of Q on the state reached after nsteps steps from rest
    (returns (dQdF, Q))."""
    S = Solver(cfg, Fext)
    states = [_oracle_state(S)]
    for _ in range(nsteps):
        S.run(1)
        states.append(_oracle_state(S))
    Q = objective(S, w)
    h = fd_steps(cfg, F_scale)
    P = streaming_matrix(cfg)
    J = state_jacobians(cfg, *states[nsteps], S.Fext, h)
    _, _, Us, UF = _split(cfg, J)
    lam = np.einsum("nc,nck->nk", w, Us).reshape(-1)
    dQdF = np.einsum("nc,ncd->nd", w, UF)
    for t in range(nsteps - 1, -1, -1):
        J = state_jacobians(cfg, *states[t], S.Fext, h)
        Ys, YF, _, _ = _split(cfg, J)
        v = (P.T @ lam).reshape(cfg.N, -1)
        dQdF += np.einsum("ni,nid->nd", v, YF)
        lam = np.einsum("ni,nik->nk", v, Ys).reshape(-1)
    return dQdF, Q


def fd_steady(cfg: Config, Fext: np.ndarray, w: np.ndarray, node: int, comp: int, h: float,
              tol: float = 1e-11, max_steps: int = 2_000_000) -> float:
    """Central difference of the steady Q in F_comp at one node (two oracle
    solves from rest)."""
    vals = []
    for sgn in (1.0, -1.0):
        F = np.array(Fext, dtype=np.float64).reshape(cfg.N, 3).copy()
        F[node, comp] += sgn * h
        vals.append(objective(steady_state(cfg, F, tol, max_steps), w))
    return (vals[0] - vals[1]) / (2.0 * h)


def fd_unrolled(cfg: Config, Fext: np.ndarray, w: np.ndarray, nsteps: int, node: int, comp: int,
                h: float) -> float:
    vals = []
    for sgn in (1.0, -1.0):
        F = np.array(Fext, dtype=np.float64).reshape(cfg.N, 3).copy()
        F[node, comp] += sgn * h
        S = Solver(cfg, F)
        S.run(nsteps)
        vals.append(objective(S, w))
    return (vals[0] - vals[1]) / (2.0 * h)
