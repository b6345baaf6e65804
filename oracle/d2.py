"""FP64 CPU oracle of the two-dimensional models: D2Q9 preconditioned GLBE
with forcing term and D2Q5 preconditioned vector lattice for the induction
(arXiv:0809.4730 Secs. 2-4, App. A D2Q9 tables).

TEST INFRASTRUCTURE ONLY, like the rest of this package: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The arithmetic lives in ``glbe_oracle2d.c`` (plain C, FP64, no FMA
contraction), compiled with gcc on first use and wrapped with ctypes.  Storage
is array-of-structures: f[N, 9], g[N, 2, 5] (component j, direction a),
FL[N, 2]; node n = y*nx + x.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.environ.get("GLBE_ORACLE2D_SOURCE") or os.path.join(_HERE, "glbe_oracle2d.c")
_BUILD_DIR = os.environ.get("GLBE_ORACLE_BUILD_DIR") or os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle2d.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``glbe_oracle2d.c`` into ``_build/liboracle2d.so`` with the
    flags of the 3D oracle (IEEE FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wno-unused-function",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params2(C.Structure):
    """Mirror of ``orc2_params`` in glbe_oracle2d.c."""
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("wall_lo", C.c_int * 2), ("wall_hi", C.c_int * 2),
        ("rho0", C.c_double), ("gamma", C.c_double), ("nu", C.c_double),
        ("s", C.c_double * 9), ("F", C.c_double * 2),
        ("induction", C.c_int),
        ("gamma_m", C.c_double), ("eta", C.c_double), ("chi", C.c_double),
        ("mu", C.c_double), ("B0", C.c_double * 2),
    ]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L = C.POINTER(C.c_long)
_P = C.POINTER(Params2)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc2_params_size.restype = C.c_int
            L.orc2_lattice.argtypes = [_I, _D, _I]
            L.orc2_moment_matrix.argtypes = [_D]
            L.orc2_equilibrium_moments.argtypes = [C.c_double, _D, C.c_double, _D]
            L.orc2_source_moments.argtypes = [_D, _D, C.c_double, _D]
            L.orc2_source_precond_diag.argtypes = [C.c_double, _D]
            L.orc2_relaxation_rates.argtypes = [_P, _D]
            L.orc2_tau_m.argtypes = [_P]
            L.orc2_tau_m.restype = C.c_double
            L.orc2_vector_equilibrium.argtypes = [_P, _D, _D, _D]
            L.orc2_current_z.argtypes = [_P, _D, _D]
            L.orc2_current_z.restype = C.c_double
            L.orc2_collide_node.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D]
            L.orc2_is_solid.argtypes = [_P, C.c_int, C.c_int]
            L.orc2_is_solid.restype = C.c_int
            L.orc2_init_state.argtypes = [_P, _D, _D, _D]
            L.orc2_fields.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D]
            L.orc2_run.argtypes = [_P, _D, _D, _D, _D, _D, _L, C.c_long, C.c_long, C.c_double, _D, C.c_long, _L]
            L.orc2_run.restype = C.c_long
            assert L.orc2_params_size() == C.sizeof(Params2), "2D oracle params layout mismatch"
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _vec(v, n):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(n))


def paper_rates() -> np.ndarray:
    """Kinetic rates of the D2Q9 model quoted in Sec. 3: s_1 = 1.63,
    s_2 = 1.14, s_4 = s_6 = 1.92; conserved rows 0, 3, 5 take 1.0 and the
    viscous rows 7, 8 are set from nu/gamma."""
    s = np.ones(9)
    s[1], s[2] = 1.63, 1.14
    s[4] = s[6] = 1.92
    return s


@dataclass
class Config2:
    """One oracle problem on an nx x ny grid."""
    nx: int
    ny: int
    wall_lo: tuple = (0, 0)
    wall_hi: tuple = (0, 0)
    rho0: float = 1.0
    gamma: float = 1.0
    nu: float = 0.1
    s: np.ndarray = field(default_factory=paper_rates)
    F: tuple = (0.0, 0.0)
    induction: bool = False
    gamma_m: float = 1.0
    eta: float = 0.1
    chi: float = 1.0
    mu: float = 1.0
    B0: tuple = (0.0, 0.0)

    def params(self) -> Params2:
        p = Params2()
        p.nx, p.ny = self.nx, self.ny
        for d in range(2):
            p.wall_lo[d] = int(self.wall_lo[d])
            p.wall_hi[d] = int(self.wall_hi[d])
            p.F[d] = float(self.F[d])
            p.B0[d] = float(self.B0[d])
        p.rho0, p.gamma, p.nu = self.rho0, self.gamma, self.nu
        for k in range(9):
            p.s[k] = float(self.s[k])
        p.induction = int(bool(self.induction))
        p.gamma_m, p.eta, p.chi, p.mu = self.gamma_m, self.eta, self.chi, self.mu
        return p

    @property
    def N(self) -> int:
        return self.nx * self.ny


def lattice():
    """(E[9,2], w[9], opp[9]) of the oracle's D2Q9 ordering."""
    E = np.zeros(18, dtype=np.int32)
    w = np.zeros(9)
    opp = np.zeros(9, dtype=np.int32)
    lib().orc2_lattice(E.ctypes.data_as(_I), _p(w), opp.ctypes.data_as(_I))
    return E.reshape(9, 2), w, opp


def moment_matrix() -> np.ndarray:
    T = np.zeros(81)
    lib().orc2_moment_matrix(_p(T))
    return T.reshape(9, 9)


def equilibrium_moments(rho, j, gamma) -> np.ndarray:
    out = np.zeros(9)
    lib().orc2_equilibrium_moments(float(rho), _p(_vec(j, 2)), float(gamma), _p(out))
    return out


def source_moments(F, u, gamma) -> np.ndarray:
    out = np.zeros(9)
    lib().orc2_source_moments(_p(_vec(F, 2)), _p(_vec(u, 2)), float(gamma), _p(out))
    return out


def source_precond_diag(gamma) -> np.ndarray:
    out = np.zeros(9)
    lib().orc2_source_precond_diag(float(gamma), _p(out))
    return out


def relaxation_rates(cfg: Config2) -> np.ndarray:
    out = np.zeros(9)
    p = cfg.params()
    lib().orc2_relaxation_rates(C.byref(p), _p(out))
    return out


def tau_m(cfg: Config2) -> float:
    p = cfg.params()
    return lib().orc2_tau_m(C.byref(p))


def vector_equilibrium(cfg: Config2, u, B) -> np.ndarray:
    """g^eq,* as [2, 5] (component j, direction a)."""
    out = np.zeros(10)
    p = cfg.params()
    lib().orc2_vector_equilibrium(C.byref(p), _p(_vec(u, 2)), _p(_vec(B, 2)), _p(out))
    return out.reshape(2, 5)


def current_z(cfg: Config2, g, geq) -> float:
    p = cfg.params()
    return lib().orc2_current_z(C.byref(p), _p(_vec(g, 10)), _p(_vec(geq, 10)))


def collide_node(cfg: Config2, f, g=None, FLprev=None, Fext=None):
    """Single-node collision: (f~[9], g~[2,5] or None, macro dict)."""
    ft, gt, mac = np.zeros(9), np.zeros(10), np.zeros(7)
    p = cfg.params()
    lib().orc2_collide_node(C.byref(p), _p(_vec(f, 9)), None if g is None else _p(_vec(g, 10)),
                            None if FLprev is None else _p(_vec(FLprev, 2)),
                            None if Fext is None else _p(_vec(Fext, 2)), _p(ft), _p(gt), _p(mac))
    return ft, (gt.reshape(2, 5) if cfg.induction else None), dict(rho=mac[0], u=mac[1:3], B=mac[3:5], FL=mac[5:7])


class Solver2:
    """Time-marching FP64 solver on the 2D lattices (oracle).  Fext is [N, 2]
    (added to the uniform F)."""

    def __init__(self, cfg: Config2, Fext: np.ndarray | None = None):
        self.cfg = cfg
        self._p = cfg.params()
        N = cfg.N
        self.f = np.zeros((N, 9))
        self.g = np.zeros((N, 2, 5)) if cfg.induction else np.zeros((1, 2, 5))
        self.FL = np.zeros((N, 2))
        self.Fext = None if Fext is None else np.ascontiguousarray(Fext, dtype=np.float64).reshape(N, 2)
        self.usnap = np.zeros((N, 2))
        self._tsnap = C.c_long(-1)
        self.t = 0
        self.hist = []
        lib().orc2_init_state(C.byref(self._p), _p(self.f), _p(self.g) if cfg.induction else None, _p(self.FL))

    def run(self, nsteps: int, tol: float = 0.0) -> int:
        cap = nsteps // 10 + 2
        h = np.zeros((cap, 8))
        nh = C.c_long(0)
        t = lib().orc2_run(C.byref(self._p), _p(self.f), _p(self.g) if self.cfg.induction else None,
                           _p(self.FL), _p(self.Fext), _p(self.usnap), C.byref(self._tsnap),
                           self.t, int(nsteps), float(tol), _p(h), cap, C.byref(nh))
        for row in h[:nh.value]:
            self.hist.append(dict(t=int(row[0]), r=row[1], num=row[2], den=row[3], mass=row[4],
                                  mom=row[5:7].copy()))
        self.t = int(t)
        return self.t

    def fields(self):
        """(rho[N], u[N,2], B[N,2]) of the current state (zero on walls)."""
        N = self.cfg.N
        rho, u, B = np.zeros(N), np.zeros((N, 2)), np.zeros((N, 2))
        lib().orc2_fields(C.byref(self._p), _p(self.f), _p(self.g) if self.cfg.induction else None,
                          _p(self.FL), _p(self.Fext), _p(rho), _p(u), _p(B))
        return rho, u, B

    def solid_mask(self) -> np.ndarray:
        return solid_mask(self.cfg)


def solid_mask(c: Config2) -> np.ndarray:
    """[N] bool: the node lies on a wall line."""
    m = np.zeros((c.ny, c.nx), dtype=bool)
    if c.wall_lo[0]:
        m[:, 0] = True
    if c.wall_hi[0]:
        m[:, -1] = True
    if c.wall_lo[1]:
        m[0, :] = True
    if c.wall_hi[1]:
        m[-1, :] = True
    return m.reshape(-1)
