"""FP64 CPU oracle of the preconditioned GLBE + D3Q7 induction lattice.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library and
its Python binding never import it, and it imports nothing from them.

The arithmetic lives in ``glbe_oracle.c`` (plain C, FP64, no FMA contraction);
this module compiles it with gcc on first use and wraps it with ctypes.  The
oracle's own storage is array-of-structures (``f[n, a]``); the helpers
``to_soa``/``from_soa`` convert to the structure-of-arrays layout
``[a][z][y][x]`` used at the C-ABI boundary of the CUDA library.

Citations are to arXiv:0809.4730 (sections, equations, appendices).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GLBE_ORACLE_SOURCE / GLBE_ORACLE_BUILD_DIR let the mutation tests build a
# deliberately broken copy of the source elsewhere (test use only).
_SRC = os.environ.get("GLBE_ORACLE_SOURCE") or os.path.join(_HERE, "glbe_oracle.c")
_BUILD_DIR = os.environ.get("GLBE_ORACLE_BUILD_DIR") or os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``glbe_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2,
    OpenMP, IEEE FP64 without FMA contraction so x86 and Arm agree bit for
    bit).  Rebuilds when the source is newer than the library."""
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


class Params(C.Structure):
    """Mirror of ``orc_params`` in glbe_oracle.c."""
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("wall_lo", C.c_int * 3), ("wall_hi", C.c_int * 3),
        ("rho0", C.c_double), ("gamma", C.c_double), ("nu", C.c_double),
        ("s", C.c_double * 19), ("F", C.c_double * 3),
        ("induction", C.c_int),
        ("gamma_m", C.c_double), ("eta", C.c_double), ("chi", C.c_double),
        ("mu", C.c_double), ("B0", C.c_double * 3),
        ("box", C.c_int), ("box_lo", C.c_int * 3), ("box_hi", C.c_int * 3),
        ("U_lid", C.c_double * 3),
    ]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L = C.POINTER(C.c_long)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.orc_params_size.restype = C.c_int
            L.orc_lattice_d3q19.argtypes = [_I, _D, _I]
            L.orc_moment_matrix.argtypes = [_D]
            L.orc_inverse_moment_matrix.argtypes = [_D]
            L.orc_equilibrium_moments.argtypes = [C.c_double, _D, C.c_double, _D]
            L.orc_source_moments.argtypes = [_D, _D, C.c_double, _D]
            L.orc_source_precond_diag.argtypes = [C.c_double, _D]
            L.orc_relaxation_rates.argtypes = [C.POINTER(Params), _D]
            L.orc_tau_m.argtypes = [C.POINTER(Params)]
            L.orc_tau_m.restype = C.c_double
            L.orc_vector_equilibrium.argtypes = [C.POINTER(Params), _D, _D, _D]
            L.orc_current_density.argtypes = [C.POINTER(Params), _D, _D, _D]
            L.orc_collide_node.argtypes = [C.POINTER(Params), _D, _D, _D, _D, _D, _D, _D]
            L.orc_is_solid.argtypes = [C.POINTER(Params), C.c_int, C.c_int, C.c_int]
            L.orc_is_solid.restype = C.c_int
            L.orc_init_state.argtypes = [C.POINTER(Params), _D, _D, _D]
            L.orc_fields.argtypes = [C.POINTER(Params), _D, _D, _D, _D, _D, _D, _D, _D]
            L.orc_run.argtypes = [C.POINTER(Params), _D, _D, _D, _D, _D, _L,
                                  C.c_long, C.c_long, C.c_double, _D, C.c_long, _L]
            L.orc_run.restype = C.c_long
            L.orc_node_jacobian.argtypes = [C.POINTER(Params), _D, _D, _D, _D, _D, _D]
            L.orc_state_jacobians.argtypes = [C.POINTER(Params), _D, _D, _D, _D, _D, _D]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            assert L.orc_params_size() == C.sizeof(Params), "oracle params layout mismatch"
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


# Kinetic relaxation rates of the D3Q19 model quoted in Sec. 3
# (s1 = 1.19, s2 = s10 = s12 = 1.4, s4 = s6 = s8 = 1.2, s16..18 = 1.98).
# The conserved rows 0, 3, 5, 7 take 1.0 (their value cannot matter).
def paper_rates() -> np.ndarray:
    s = np.ones(19)
    s[1] = 1.19
    s[2] = s[10] = s[12] = 1.4
    s[4] = s[6] = s[8] = 1.2
    s[16] = s[17] = s[18] = 1.98
    return s


@dataclass
class Config:
    """Plain description of one oracle problem."""
    nx: int
    ny: int
    nz: int
    wall_lo: tuple = (0, 0, 0)
    wall_hi: tuple = (0, 0, 0)
    rho0: float = 1.0
    gamma: float = 1.0
    nu: float = 0.1
    s: np.ndarray = field(default_factory=paper_rates)
    F: tuple = (0.0, 0.0, 0.0)
    induction: bool = False
    gamma_m: float = 1.0
    eta: float = 0.1
    chi: float = 1.0
    mu: float = 1.0
    B0: tuple = (0.0, 0.0, 0.0)
    box: tuple | None = None       # ((lo_x, lo_y, lo_z), (hi_x, hi_y, hi_z)): fluid box of the flow lattice
    U_lid: tuple = (0.0, 0.0, 0.0)  # velocity of the boundary above the highest fluid z plane

    def params(self) -> Params:
        p = Params()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        for d in range(3):
            p.wall_lo[d] = int(self.wall_lo[d])
            p.wall_hi[d] = int(self.wall_hi[d])
            p.F[d] = float(self.F[d])
            p.B0[d] = float(self.B0[d])
        p.rho0, p.gamma, p.nu = self.rho0, self.gamma, self.nu
        for k in range(19):
            p.s[k] = float(self.s[k])
        p.induction = int(bool(self.induction))
        p.gamma_m, p.eta, p.chi, p.mu = self.gamma_m, self.eta, self.chi, self.mu
        p.box = int(self.box is not None)
        for d in range(3):
            p.box_lo[d] = int(self.box[0][d]) if self.box is not None else 0
            p.box_hi[d] = int(self.box[1][d]) if self.box is not None else 0
            p.U_lid[d] = float(self.U_lid[d])
        return p

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz


def lattice():
    """(E[19,3], w[19], opp[19]) of the oracle's D3Q19 ordering."""
    E = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, dtype=np.int32)
    lib().orc_lattice_d3q19(E.ctypes.data_as(_I), _p(w), opp.ctypes.data_as(_I))
    return E.reshape(19, 3), w, opp


def moment_matrix() -> np.ndarray:
    T = np.zeros(19 * 19)
    lib().orc_moment_matrix(_p(T))
    return T.reshape(19, 19)


def inverse_moment_matrix() -> np.ndarray:
    T = np.zeros(19 * 19)
    lib().orc_inverse_moment_matrix(_p(T))
    return T.reshape(19, 19)


def equilibrium_moments(rho: float, j, gamma: float) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_equilibrium_moments(float(rho), _p(np.asarray(j, dtype=np.float64).copy()), float(gamma), _p(out))
    return out


def source_moments(F, u, gamma: float) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_source_moments(_p(np.asarray(F, dtype=np.float64).copy()),
                             _p(np.asarray(u, dtype=np.float64).copy()), float(gamma), _p(out))
    return out


def source_precond_diag(gamma: float) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_source_precond_diag(float(gamma), _p(out))
    return out


def relaxation_rates(cfg: Config) -> np.ndarray:
    out = np.zeros(19)
    p = cfg.params()
    lib().orc_relaxation_rates(C.byref(p), _p(out))
    return out


def tau_m(cfg: Config) -> float:
    p = cfg.params()
    return lib().orc_tau_m(C.byref(p))


def vector_equilibrium(cfg: Config, u, B) -> np.ndarray:
    """g^eq,* as [3, 7] (component j, direction a)."""
    out = np.zeros(21)
    p = cfg.params()
    lib().orc_vector_equilibrium(C.byref(p), _p(np.asarray(u, dtype=np.float64).copy()),
                                 _p(np.asarray(B, dtype=np.float64).copy()), _p(out))
    return out.reshape(3, 7)


def current_density(cfg: Config, g, geq) -> np.ndarray:
    out = np.zeros(3)
    p = cfg.params()
    lib().orc_current_density(C.byref(p), _p(np.ascontiguousarray(g, dtype=np.float64).reshape(21)),
                              _p(np.ascontiguousarray(geq, dtype=np.float64).reshape(21)), _p(out))
    return out


def collide_node(cfg: Config, f, g=None, FLprev=None, Fext=None):
    """Single-node collision: returns (f~[19], g~[21] or None, macro dict)."""
    ft = np.zeros(19)
    gt = np.zeros(21)
    mac = np.zeros(10)
    p = cfg.params()
    f = np.ascontiguousarray(f, dtype=np.float64)
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64).reshape(21)
    fl = None if FLprev is None else np.ascontiguousarray(FLprev, dtype=np.float64)
    fe = None if Fext is None else np.ascontiguousarray(Fext, dtype=np.float64)
    lib().orc_collide_node(C.byref(p), _p(f), _p(gg), _p(fl), _p(fe), _p(ft), _p(gt), _p(mac))
    return ft, (gt if cfg.induction else None), dict(rho=mac[0], u=mac[1:4], B=mac[4:7], FL=mac[7:10])


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return lib().orc_get_threads()


class Solver:
    """Time-marching FP64 solver (oracle).  State arrays are AoS:
    f[N,19], g[N,3,7], FL[N,3]; Fext is [N,3] (added to the uniform F)."""

    def __init__(self, cfg: Config, Fext: np.ndarray | None = None):
        self.cfg = cfg
        self._p = cfg.params()
        N = cfg.N
        self.f = np.zeros((N, 19))
        self.g = np.zeros((N, 3, 7)) if cfg.induction else np.zeros((1, 3, 7))
        self.FL = np.zeros((N, 3))
        self.Fext = None if Fext is None else np.ascontiguousarray(Fext, dtype=np.float64).reshape(N, 3)
        self.usnap = np.zeros((N, 3))
        self._tsnap = C.c_long(-1)
        self.t = 0
        self.hist = []
        lib().orc_init_state(C.byref(self._p), _p(self.f),
                             _p(self.g) if cfg.induction else None, _p(self.FL))

    def run(self, nsteps: int, tol: float = 0.0) -> int:
        cap = nsteps // 10 + 2
        h = np.zeros((cap, 8))
        nh = C.c_long(0)
        t = lib().orc_run(C.byref(self._p), _p(self.f), _p(self.g) if self.cfg.induction else None,
                          _p(self.FL), _p(self.Fext), _p(self.usnap), C.byref(self._tsnap),
                          self.t, int(nsteps), float(tol), _p(h), cap, C.byref(nh))
        for row in h[:nh.value]:
            self.hist.append(dict(t=int(row[0]), r=row[1], num=row[2], den=row[3], mass=row[4],
                                  mom=row[5:8].copy()))
        self.t = int(t)
        return self.t

    def fields(self):
        """(rho[N], u[N,3], B[N,3], FL_next[N,3]) of the current state."""
        N = self.cfg.N
        rho = np.zeros(N)
        u = np.zeros((N, 3))
        B = np.zeros((N, 3))
        FLn = np.zeros((N, 3))
        lib().orc_fields(C.byref(self._p), _p(self.f), _p(self.g) if self.cfg.induction else None,
                         _p(self.FL), _p(self.Fext), _p(rho), _p(u), _p(B), _p(FLn))
        return rho, u, B, FLn

    def solid_mask(self) -> np.ndarray:
        return solid_mask(self.cfg)


def solid_mask(c: Config) -> np.ndarray:
    """[N] bool: the node is not fluid for the flow lattice (on a wall plane,
    or outside the fluid box)."""
    m = np.zeros((c.nz, c.ny, c.nx), dtype=bool)
    if c.box is not None:
        (lx, ly, lz), (hx, hy, hz) = c.box
        inside = np.zeros_like(m)
        inside[lz:hz + 1, ly:hy + 1, lx:hx + 1] = True
        m |= ~inside
    for d, n in zip(range(3), (c.nx, c.ny, c.nz)):
        sl = [slice(None)] * 3
        if c.wall_lo[d]:
            sl[2 - d] = 0
            m[tuple(sl)] = True
        if c.wall_hi[d]:
            sl[2 - d] = n - 1
            m[tuple(sl)] = True
    return m.reshape(-1)


# ---------------------------------------------------------------------------
# Layout conversion to/from the C-ABI layout [component][z][y][x].
# ---------------------------------------------------------------------------
def to_soa(a: np.ndarray) -> np.ndarray:
    """[N, q] or [N, 3, 7] (AoS) -> [q, N] (SoA); g keeps (j, a) order."""
    N = a.shape[0]
    return np.ascontiguousarray(a.reshape(N, -1).T)


def from_soa(a: np.ndarray, shape_tail) -> np.ndarray:
    q = a.shape[0]
    return np.ascontiguousarray(a.reshape(q, -1).T).reshape((-1,) + tuple(shape_tail))
