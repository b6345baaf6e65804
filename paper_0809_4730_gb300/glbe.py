"""Python binding of the C-ABI in include/glbe.h and include/glbe2d.h
(argument marshalling only).

Every step of the time march runs in the CUDA library ``libglbe.so``; this
module loads it with ctypes, mirrors its structs and exposes the entry points
under the same names.  PyTorch provides device memory (the caller-owned
workspace and field buffers) and the CUDA stream.

There is no fallback: if the library is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

GLBE_OK, GLBE_ERR_ARG, GLBE_ERR_CUDA, GLBE_ERR_DIVERGED, GLBE_ERR_TIMEOUT, GLBE_ERR_STATE = range(6)
GLBE_F32, GLBE_BF16, GLBE_F16, GLBE_F32C, GLBE_BF16_SR, GLBE_F16_SR = 0, 1, 2, 3, 4, 5
STORAGE = {"f32": GLBE_F32, "bf16": GLBE_BF16, "f16": GLBE_F16, "f32c": GLBE_F32C, "bf16sr": GLBE_BF16_SR,
           "f16sr": GLBE_F16_SR}


class GlbeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class glbe_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("wall_lo", C.c_int * 3), ("wall_hi", C.c_int * 3),
        ("rho0", C.c_double), ("gamma", C.c_double), ("nu", C.c_double),
        ("s", C.c_double * 19), ("F", C.c_double * 3),
        ("force_field", C.c_int), ("induction", C.c_int),
        ("gamma_m", C.c_double), ("eta", C.c_double), ("chi", C.c_double), ("mu", C.c_double),
        ("B0", C.c_double * 3),
        ("storage", C.c_int), ("storage_scale", C.c_double),
        ("stream", C.c_void_p),
        ("variant", C.c_int),
        ("collision", C.c_int),
        ("box", C.c_int), ("box_lo", C.c_int * 3), ("box_hi", C.c_int * 3), ("U_lid", C.c_double * 3),
        ("ghost_lo", C.c_int), ("ghost_hi", C.c_int),
    ]


class glbe_residual_info(C.Structure):
    _fields_ = [
        ("t", C.c_long), ("r", C.c_double), ("num", C.c_double), ("den", C.c_double),
        ("mass", C.c_double), ("momentum", C.c_double * 3), ("nonfinite", C.c_int),
    ]


class glbe_batch_result(C.Structure):
    _fields_ = [("converged", C.c_int), ("steps", C.c_long), ("r", C.c_double), ("seconds", C.c_double),
                ("nonfinite", C.c_int)]


class glbe2d_params(C.Structure):
    """Mirror of glbe2d_params (include/glbe2d.h)."""
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("wall_lo", C.c_int * 2), ("wall_hi", C.c_int * 2),
        ("rho0", C.c_double), ("gamma", C.c_double), ("nu", C.c_double),
        ("s", C.c_double * 9), ("F", C.c_double * 2),
        ("force_field", C.c_int), ("induction", C.c_int),
        ("gamma_m", C.c_double), ("eta", C.c_double), ("chi", C.c_double), ("mu", C.c_double),
        ("B0", C.c_double * 2),
        ("storage", C.c_int),
        ("stream", C.c_void_p),
        ("variant", C.c_int),
    ]


# Every symbol include/glbe.h and include/glbe2d.h declare, with (restype, argtypes).
_P = C.POINTER
_SIGNATURES = {
    "glbe_params_default": (None, [_P(glbe_params)]),
    "glbe_workspace_bytes": (C.c_int, [_P(glbe_params), _P(C.c_size_t)]),
    "glbe_init": (C.c_int, [_P(glbe_params), C.c_void_p, C.c_size_t, _P(C.c_void_p)]),
    "glbe_set_force": (C.c_int, [C.c_void_p, C.c_void_p]),
    "glbe_set_force_host": (C.c_int, [C.c_void_p, C.c_void_p]),
    "glbe_step_n": (C.c_int, [C.c_void_p, C.c_long]),
    "glbe_residual": (C.c_int, [C.c_void_p, _P(glbe_residual_info)]),
    "glbe_history": (C.c_int, [C.c_void_p, _P(glbe_residual_info), C.c_long, _P(C.c_long)]),
    "glbe_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_long, _P(C.c_long), _P(C.c_double)]),
    "glbe_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "glbe_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "glbe_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_long]),
    "glbe_time": (C.c_int, [C.c_void_p, _P(C.c_long)]),
    "glbe_sync": (C.c_int, [C.c_void_p]),
    "glbe_last_error": (C.c_char_p, []),
    "glbe_destroy": (None, [C.c_void_p]),
    "glbe_abi_version": (C.c_int, []),
    "glbe_struct_sizes": (None, [_P(C.c_size_t), _P(C.c_size_t)]),
    "glbe_batch_workspace_bytes": (C.c_int, [_P(glbe_params), C.c_int, _P(C.c_size_t)]),
    "glbe_batch_init": (C.c_int, [_P(glbe_params), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p, _P(C.c_void_p)]),
    "glbe_batch_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "glbe_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, _P(C.c_int), _P(C.c_int), _P(C.c_double)]),
    "glbe_batch_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_long, C.c_int, _P(glbe_batch_result),
                                   _P(C.c_double)]),
    "glbe_batch_fields": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "glbe_batch_reset": (C.c_int, [C.c_void_p]),
    "glbe_batch_set_barrier_test": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int]),
    "glbe_batch_destroy": (None, [C.c_void_p]),
    "glbe_step_residual_noalloc": (C.c_int, [_P(glbe_params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_int, C.c_long, _P(glbe_residual_info)]),
    "glbe_halo_bytes": (C.c_int, [C.c_void_p, _P(C.c_size_t)]),
    "glbe_halo_pack": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "glbe_halo_unpack": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "glbe_residual_combine": (C.c_int, [_P(glbe_residual_info), C.c_int, _P(glbe_residual_info)]),
    "glbe_checkpoint_bytes": (C.c_int, [C.c_void_p, _P(C.c_size_t)]),
    "glbe_checkpoint_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "glbe_checkpoint_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "glbe_adjoint_workspace_bytes": (C.c_int, [_P(glbe_params), C.c_long, C.c_long, _P(C.c_size_t)]),
    "glbe_adjoint_steady": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_long, C.c_void_p, C.c_size_t,
                                      C.c_void_p, _P(C.c_long), _P(C.c_double)]),
    "glbe_adjoint_unrolled": (C.c_int, [C.c_void_p, C.c_void_p, C.c_long, C.c_long, C.c_void_p, C.c_size_t,
                                        C.c_void_p]),
    "glbe2d_params_default": (None, [_P(glbe2d_params)]),
    "glbe2d_workspace_bytes": (C.c_int, [_P(glbe2d_params), _P(C.c_size_t)]),
    "glbe2d_init": (C.c_int, [_P(glbe2d_params), C.c_void_p, C.c_size_t, _P(C.c_void_p)]),
    "glbe2d_set_force": (C.c_int, [C.c_void_p, C.c_void_p]),
    "glbe2d_step_n": (C.c_int, [C.c_void_p, C.c_long]),
    "glbe2d_residual": (C.c_int, [C.c_void_p, _P(glbe_residual_info)]),
    "glbe2d_history": (C.c_int, [C.c_void_p, _P(glbe_residual_info), C.c_long, _P(C.c_long)]),
    "glbe2d_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_long, _P(C.c_long), _P(C.c_double)]),
    "glbe2d_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "glbe2d_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "glbe2d_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_long]),
    "glbe2d_time": (C.c_int, [C.c_void_p, _P(C.c_long)]),
    "glbe2d_sync": (C.c_int, [C.c_void_p]),
    "glbe2d_destroy": (None, [C.c_void_p]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libglbe.so (building it with nvcc if it is absent or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run paper_0809_4730_gb300.build.build()")
            lib = C.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            if lib.glbe_abi_version() != 4:
                raise RuntimeError("libglbe ABI version mismatch")
            ps, isz = C.c_size_t(0), C.c_size_t(0)
            lib.glbe_struct_sizes(C.byref(ps), C.byref(isz))
            if ps.value != C.sizeof(glbe_params) or isz.value != C.sizeof(glbe_residual_info):
                raise RuntimeError("libglbe struct layout does not match the Python mirror")
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != GLBE_OK:
        msg = load().glbe_last_error().decode(errors="replace")
        raise GlbeError(status, where, msg)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# Same-name wrappers of the C entry points
# ---------------------------------------------------------------------------
def glbe_params_default() -> glbe_params:
    p = glbe_params()
    load().glbe_params_default(C.byref(p))
    return p


def glbe_workspace_bytes(p: glbe_params) -> int:
    n = C.c_size_t(0)
    _check(load().glbe_workspace_bytes(C.byref(p), C.byref(n)), "glbe_workspace_bytes")
    return n.value


def glbe_init(p: glbe_params, workspace) -> C.c_void_p:
    ctx = C.c_void_p()
    _check(load().glbe_init(C.byref(p), _ptr(workspace), workspace.numel() * workspace.element_size(),
                            C.byref(ctx)), "glbe_init")
    return ctx


def glbe_set_force(ctx, d_F):
    _check(load().glbe_set_force(ctx, _ptr(d_F)), "glbe_set_force")


def glbe_set_force_host(ctx, h_F):
    _check(load().glbe_set_force_host(ctx, _ptr(h_F)), "glbe_set_force_host")


def glbe_step_n(ctx, n: int):
    _check(load().glbe_step_n(ctx, int(n)), "glbe_step_n")


def glbe_residual(ctx) -> glbe_residual_info:
    info = glbe_residual_info()
    _check(load().glbe_residual(ctx, C.byref(info)), "glbe_residual")
    return info


def glbe_history(ctx, cap: int = 4096):
    buf = (glbe_residual_info * int(cap))()
    n = C.c_long(0)
    _check(load().glbe_history(ctx, buf, int(cap), C.byref(n)), "glbe_history")
    return [dict(t=buf[i].t, r=buf[i].r, num=buf[i].num, den=buf[i].den, mass=buf[i].mass,
                 momentum=tuple(buf[i].momentum), nonfinite=buf[i].nonfinite) for i in range(n.value)]


def glbe_solve(ctx, tol: float, max_steps: int):
    steps = C.c_long(0)
    r = C.c_double(0.0)
    st = load().glbe_solve(ctx, float(tol), int(max_steps), C.byref(steps), C.byref(r))
    if st not in (GLBE_OK, GLBE_ERR_TIMEOUT):
        _check(st, "glbe_solve")
    return st, steps.value, r.value


def glbe_fields(ctx, d_rho, d_u, d_B):
    _check(load().glbe_fields(ctx, _ptr(d_rho), _ptr(d_u), _ptr(d_B)), "glbe_fields")


def glbe_get_state(ctx, d_df, d_dg, d_FL):
    _check(load().glbe_get_state(ctx, _ptr(d_df), _ptr(d_dg), _ptr(d_FL)), "glbe_get_state")


def glbe_set_state(ctx, d_df, d_dg, d_FL, t: int):
    _check(load().glbe_set_state(ctx, _ptr(d_df), _ptr(d_dg), _ptr(d_FL), int(t)), "glbe_set_state")


def glbe_time(ctx) -> int:
    t = C.c_long(0)
    _check(load().glbe_time(ctx, C.byref(t)), "glbe_time")
    return t.value


def glbe_sync(ctx):
    _check(load().glbe_sync(ctx), "glbe_sync")


def glbe_step_residual_noalloc(p: glbe_params, d_src, d_dst, d_force, d_u, have_prev: bool, t: int):
    """One fused time step with the residual on caller-held buffers; no device
    memory is allocated (see include/glbe.h).  Returns glbe_residual_info."""
    info = glbe_residual_info()
    _check(load().glbe_step_residual_noalloc(C.byref(p), _ptr(d_src), _ptr(d_dst), _ptr(d_force), _ptr(d_u),
                                             int(bool(have_prev)), int(t), C.byref(info)),
           "glbe_step_residual_noalloc")
    return info


def glbe_halo_bytes(ctx) -> int:
    n = C.c_size_t(0)
    _check(load().glbe_halo_bytes(ctx, C.byref(n)), "glbe_halo_bytes")
    return n.value


def glbe_halo_pack(ctx, face: int, d_buf):
    _check(load().glbe_halo_pack(ctx, int(face), _ptr(d_buf)), "glbe_halo_pack")


def glbe_halo_unpack(ctx, face: int, d_buf):
    _check(load().glbe_halo_unpack(ctx, int(face), _ptr(d_buf)), "glbe_halo_unpack")


def glbe_residual_combine(parts) -> glbe_residual_info:
    """Record of a grid from the records of its slabs (host only, no device)."""
    arr = (glbe_residual_info * len(parts))(*parts)
    out = glbe_residual_info()
    _check(load().glbe_residual_combine(arr, len(parts), C.byref(out)), "glbe_residual_combine")
    return out


def glbe_destroy(ctx):
    if ctx:
        load().glbe_destroy(ctx)


def glbe_checkpoint_bytes(ctx) -> int:
    n = C.c_size_t(0)
    _check(load().glbe_checkpoint_bytes(ctx, C.byref(n)), "glbe_checkpoint_bytes")
    return n.value


def glbe_checkpoint_save(ctx) -> bytes:
    """The context's raw state as a bytes object (see include/glbe.h)."""
    n = glbe_checkpoint_bytes(ctx)
    buf = C.create_string_buffer(n)
    _check(load().glbe_checkpoint_save(ctx, buf, n), "glbe_checkpoint_save")
    return buf.raw


def glbe_checkpoint_load(ctx, data: bytes):
    buf = C.create_string_buffer(bytes(data), len(data))
    _check(load().glbe_checkpoint_load(ctx, buf, len(data)), "glbe_checkpoint_load")


def glbe_adjoint_workspace_bytes(p: glbe_params, nsteps: int = 0, K: int = 1) -> int:
    n = C.c_size_t(0)
    _check(load().glbe_adjoint_workspace_bytes(C.byref(p), int(nsteps), int(K), C.byref(n)),
           "glbe_adjoint_workspace_bytes")
    return n.value


def glbe_adjoint_steady(ctx, d_w, tol: float, max_iters: int, work, d_dQdF):
    """Returns (status, iterations, r); status GLBE_OK or GLBE_ERR_TIMEOUT."""
    it = C.c_long(0)
    r = C.c_double(0.0)
    st = load().glbe_adjoint_steady(ctx, _ptr(d_w), float(tol), int(max_iters), _ptr(work),
                                    work.numel() * work.element_size(), _ptr(d_dQdF), C.byref(it), C.byref(r))
    if st not in (GLBE_OK, GLBE_ERR_TIMEOUT):
        _check(st, "glbe_adjoint_steady")
    return st, it.value, r.value


def glbe_adjoint_unrolled(ctx, d_w, nsteps: int, K: int, work, d_dQdF):
    _check(load().glbe_adjoint_unrolled(ctx, _ptr(d_w), int(nsteps), int(K), _ptr(work),
                                        work.numel() * work.element_size(), _ptr(d_dQdF)),
           "glbe_adjoint_unrolled")


# -- two-dimensional lattices (include/glbe2d.h) ------------------------------
def glbe2d_params_default() -> glbe2d_params:
    p = glbe2d_params()
    load().glbe2d_params_default(C.byref(p))
    return p


def glbe2d_workspace_bytes(p: glbe2d_params) -> int:
    n = C.c_size_t(0)
    _check(load().glbe2d_workspace_bytes(C.byref(p), C.byref(n)), "glbe2d_workspace_bytes")
    return n.value


def glbe2d_init(p: glbe2d_params, workspace) -> C.c_void_p:
    ctx = C.c_void_p()
    _check(load().glbe2d_init(C.byref(p), _ptr(workspace), workspace.numel() * workspace.element_size(),
                              C.byref(ctx)), "glbe2d_init")
    return ctx


def glbe2d_set_force(ctx, d_F):
    _check(load().glbe2d_set_force(ctx, _ptr(d_F)), "glbe2d_set_force")


def glbe2d_step_n(ctx, n: int):
    _check(load().glbe2d_step_n(ctx, int(n)), "glbe2d_step_n")


def glbe2d_residual(ctx) -> glbe_residual_info:
    info = glbe_residual_info()
    _check(load().glbe2d_residual(ctx, C.byref(info)), "glbe2d_residual")
    return info


def glbe2d_history(ctx, cap: int = 4096):
    arr = (glbe_residual_info * cap)()
    n = C.c_long(0)
    _check(load().glbe2d_history(ctx, arr, cap, C.byref(n)), "glbe2d_history")
    return [arr[i] for i in range(n.value)]


def glbe2d_solve(ctx, tol: float, max_steps: int):
    """Returns (status, steps, r); GLBE_ERR_TIMEOUT is returned, not raised."""
    steps, r = C.c_long(0), C.c_double(0.0)
    st = load().glbe2d_solve(ctx, float(tol), int(max_steps), C.byref(steps), C.byref(r))
    if st not in (GLBE_OK, GLBE_ERR_TIMEOUT):
        _check(st, "glbe2d_solve")
    return st, steps.value, r.value


def glbe2d_fields(ctx, d_rho, d_u, d_B):
    _check(load().glbe2d_fields(ctx, _ptr(d_rho), _ptr(d_u), _ptr(d_B)), "glbe2d_fields")


def glbe2d_get_state(ctx, d_df, d_dg, d_FL):
    _check(load().glbe2d_get_state(ctx, _ptr(d_df), _ptr(d_dg), _ptr(d_FL)), "glbe2d_get_state")


def glbe2d_set_state(ctx, d_df, d_dg, d_FL, t: int):
    _check(load().glbe2d_set_state(ctx, _ptr(d_df), _ptr(d_dg), _ptr(d_FL), int(t)), "glbe2d_set_state")


def glbe2d_time(ctx) -> int:
    t = C.c_long(0)
    _check(load().glbe2d_time(ctx, C.byref(t)), "glbe2d_time")
    return t.value


def glbe2d_sync(ctx):
    _check(load().glbe2d_sync(ctx), "glbe2d_sync")


def glbe2d_destroy(ctx):
    if ctx:
        load().glbe2d_destroy(ctx)


def make_params2d(nx, ny, **kw) -> glbe2d_params:
    """glbe2d_params from keyword arguments named as its fields (storage may
    be "f32", "bf16" or "f32c"; s overrides the 9 rates)."""
    p = glbe2d_params_default()
    p.nx, p.ny = int(nx), int(ny)
    for key, val in kw.items():
        if key in ("wall_lo", "wall_hi", "F", "B0"):
            arr = getattr(p, key)
            for d in range(2):
                arr[d] = type(arr[d])(val[d])
        elif key == "s":
            for k in range(9):
                p.s[k] = float(val[k])
        elif key == "storage":
            p.storage = STORAGE[val] if isinstance(val, str) else int(val)
        elif key in ("induction", "force_field", "variant"):
            setattr(p, key, int(val))
        else:
            setattr(p, key, float(val))
    return p


class Solver2D:
    """One D2Q9 (+ D2Q5) lattice context on a CUDA device; keyword arguments
    as the fields of ``glbe2d_params``."""

    def __init__(self, nx, ny, *, device="cuda", stream=None, **kw):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        p = make_params2d(nx, ny, **kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p.stream = C.c_void_p(self.stream.cuda_stream)
        self.params = p
        self.N = p.nx * p.ny
        self.workspace = torch.empty(glbe2d_workspace_bytes(p), dtype=torch.uint8, device=self.device)
        self.ctx = glbe2d_init(p, self.workspace)

    def close(self):
        if getattr(self, "ctx", None):
            glbe2d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def induction(self) -> bool:
        return bool(self.params.induction)

    def set_force(self, F):
        glbe2d_set_force(self.ctx, F.contiguous())

    def step(self, n: int):
        glbe2d_step_n(self.ctx, n)

    def residual(self) -> glbe_residual_info:
        return glbe2d_residual(self.ctx)

    def history(self, cap: int = 4096):
        return glbe2d_history(self.ctx, cap)

    def solve(self, tol: float, max_steps: int):
        return glbe2d_solve(self.ctx, tol, max_steps)

    @property
    def t(self) -> int:
        return glbe2d_time(self.ctx)

    def fields(self):
        torch = self.torch
        rho = torch.empty(self.N, dtype=torch.float32, device=self.device)
        u = torch.empty(2, self.N, dtype=torch.float32, device=self.device)
        B = torch.empty(2, self.N, dtype=torch.float32, device=self.device) if self.induction else None
        glbe2d_fields(self.ctx, rho, u, B)
        return rho, u, B

    def get_state(self):
        torch = self.torch
        df = torch.empty(9, self.N, dtype=torch.float32, device=self.device)
        dg = torch.empty(10, self.N, dtype=torch.float32, device=self.device) if self.induction else None
        FL = torch.empty(2, self.N, dtype=torch.float32, device=self.device) if self.induction else None
        glbe2d_get_state(self.ctx, df, dg, FL)
        return df, dg, FL

    def set_state(self, df, dg=None, FL=None, t: int = 0):
        glbe2d_set_state(self.ctx, df.contiguous(), None if dg is None else dg.contiguous(),
                         None if FL is None else FL.contiguous(), t)

    def sync(self):
        glbe2d_sync(self.ctx)


def make_params(nx, ny, nz, **kw) -> glbe_params:
    """glbe_params from keyword arguments named as its fields (storage may be
    "f32", "bf16", "f16" or "f32c"; s overrides the 19 rates)."""
    p = glbe_params_default()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    for key, val in kw.items():
        if key in ("wall_lo", "wall_hi", "F", "B0", "U_lid"):
            arr = getattr(p, key)
            for d in range(3):
                arr[d] = type(arr[d])(val[d])
        elif key == "box":
            p.box = int(val is not None)
            for d in range(3):
                p.box_lo[d] = int(val[0][d]) if val is not None else 0
                p.box_hi[d] = int(val[1][d]) if val is not None else 0
        elif key == "s":
            for k in range(19):
                p.s[k] = float(val[k])
        elif key == "storage":
            p.storage = STORAGE[val] if isinstance(val, str) else int(val)
        elif key in ("induction", "force_field", "variant", "ghost_lo", "ghost_hi", "collision"):
            setattr(p, key, int(val))
        else:
            setattr(p, key, float(val))
    return p


class Batch:
    """Many independent steady solves in one persistent launch (see
    glbe_batch_* in include/glbe.h).  domains: list of glbe_params."""

    def __init__(self, domains, *, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.n = len(domains)
        self.domains = domains
        arr = (glbe_params * self.n)(*domains)
        self._arr = arr
        nb = C.c_size_t(0)
        _check(load().glbe_batch_workspace_bytes(arr, self.n, C.byref(nb)), "glbe_batch_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        self.ptr = C.c_void_p()
        _check(load().glbe_batch_init(arr, self.n, _ptr(self.workspace), nb.value,
                                      C.c_void_p(self.stream.cuda_stream), C.byref(self.ptr)), "glbe_batch_init")

    def close(self):
        if getattr(self, "ptr", None):
            load().glbe_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_launch(self, block_threads: int, blocks_per_sm: int):
        _check(load().glbe_batch_set_launch(self.ptr, int(block_threads), int(blocks_per_sm)),
               "glbe_batch_set_launch")

    def autotune(self, steps_per_trial: int = 20):
        bt, bps, sps = C.c_int(0), C.c_int(0), C.c_double(0.0)
        _check(load().glbe_batch_autotune(self.ptr, int(steps_per_trial), C.byref(bt), C.byref(bps), C.byref(sps)),
               "glbe_batch_autotune")
        return bt.value, bps.value, sps.value

    def solve(self, tol: float, max_steps: int, use_graph: bool = True):
        res = (glbe_batch_result * self.n)()
        sec = C.c_double(0.0)
        st = load().glbe_batch_solve(self.ptr, float(tol), int(max_steps), int(bool(use_graph)), res,
                                     C.byref(sec))
        if st not in (GLBE_OK, GLBE_ERR_TIMEOUT, GLBE_ERR_DIVERGED):
            _check(st, "glbe_batch_solve")
        out = [dict(converged=bool(r.converged), steps=r.steps, r=r.r, seconds=r.seconds,
                    nonfinite=bool(r.nonfinite)) for r in res]
        return st, out, sec.value

    def fields(self, d: int):
        torch = self.torch
        p = self.domains[d]
        N = p.nx * p.ny * p.nz
        rho = torch.empty(N, dtype=torch.float32, device=self.device)
        u = torch.empty(3, N, dtype=torch.float32, device=self.device)
        B = torch.empty(3, N, dtype=torch.float32, device=self.device) if p.induction else None
        _check(load().glbe_batch_fields(self.ptr, int(d), _ptr(rho), _ptr(u), _ptr(B)), "glbe_batch_fields")
        return rho, u, B

    def reset(self):
        _check(load().glbe_batch_reset(self.ptr), "glbe_batch_reset")

    def set_barrier_test(self, spin_limit: int, absent_block: int):
        _check(load().glbe_batch_set_barrier_test(self.ptr, int(spin_limit), int(absent_block)),
               "glbe_batch_set_barrier_test")


# ---------------------------------------------------------------------------
# Convenience owner of one context and its torch-allocated workspace
# ---------------------------------------------------------------------------
class Solver:
    """One lattice context on a CUDA device.

    Keyword arguments map one to one onto the fields of ``glbe_params``;
    ``storage`` accepts "f32", "bf16" or "f16"; ``s`` overrides the 19 rates.
    """

    def __init__(self, nx, ny, nz, *, device="cuda", stream=None, **kw):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        p = glbe_params_default()
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        for key, val in kw.items():
            if key in ("wall_lo", "wall_hi", "F", "B0", "U_lid"):
                arr = getattr(p, key)
                for d in range(3):
                    arr[d] = type(arr[d])(val[d])
            elif key == "box":
                p.box = int(val is not None)
                for d in range(3):
                    p.box_lo[d] = int(val[0][d]) if val is not None else 0
                    p.box_hi[d] = int(val[1][d]) if val is not None else 0
            elif key == "s":
                for k in range(19):
                    p.s[k] = float(val[k])
            elif key == "storage":
                p.storage = STORAGE[val] if isinstance(val, str) else int(val)
            elif key in ("induction", "force_field", "variant", "ghost_lo", "ghost_hi", "collision"):
                setattr(p, key, int(val))
            else:
                setattr(p, key, float(val))
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p.stream = C.c_void_p(self.stream.cuda_stream)
        self.params = p
        self.N = p.nx * p.ny * p.nz
        nbytes = glbe_workspace_bytes(p)
        # 256-byte aligned workspace (the caching allocator aligns to 512 bytes)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = glbe_init(p, self.workspace)

    def close(self):
        if getattr(self, "ctx", None):
            glbe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def induction(self) -> bool:
        return bool(self.params.induction)

    def set_force(self, F):
        glbe_set_force(self.ctx, F.contiguous())

    def step(self, n: int):
        glbe_step_n(self.ctx, n)

    def residual(self) -> glbe_residual_info:
        return glbe_residual(self.ctx)

    def solve(self, tol: float, max_steps: int):
        return glbe_solve(self.ctx, tol, max_steps)

    def history(self, cap: int = 4096):
        return glbe_history(self.ctx, cap)

    @property
    def t(self) -> int:
        return glbe_time(self.ctx)

    def fields(self):
        torch = self.torch
        rho = torch.empty(self.N, dtype=torch.float32, device=self.device)
        u = torch.empty(3, self.N, dtype=torch.float32, device=self.device)
        B = torch.empty(3, self.N, dtype=torch.float32, device=self.device) if self.induction else None
        glbe_fields(self.ctx, rho, u, B)
        return rho, u, B

    def get_state(self):
        torch = self.torch
        df = torch.empty(19, self.N, dtype=torch.float32, device=self.device)
        dg = torch.empty(21, self.N, dtype=torch.float32, device=self.device) if self.induction else None
        FL = torch.empty(3, self.N, dtype=torch.float32, device=self.device) if self.induction else None
        glbe_get_state(self.ctx, df, dg, FL)
        return df, dg, FL

    def set_state(self, df, dg=None, FL=None, t: int = 0):
        glbe_set_state(self.ctx, df.contiguous(), None if dg is None else dg.contiguous(),
                       None if FL is None else FL.contiguous(), t)

    def sync(self):
        glbe_sync(self.ctx)

    def checkpoint(self) -> bytes:
        """Raw state for a bit-exact resume (glbe_checkpoint_save)."""
        return glbe_checkpoint_save(self.ctx)

    def restore(self, data: bytes):
        glbe_checkpoint_load(self.ctx, data)

    # -- gradients of Q = sum w . u with respect to the force field ----------
    def _adjoint_work(self, nsteps: int, K: int):
        nbytes = glbe_adjoint_workspace_bytes(self.params, nsteps, K)
        key = (nsteps, K)
        if getattr(self, "_adj_key", None) != key:
            self._adj_work = None
            self._adj_work = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)
            self._adj_key = key
        return self._adj_work

    def adjoint_steady(self, w=None, tol: float = 1e-6, max_iters: int = 1_000_000):
        """dQ/dF [3, N] at the current (steady) state; w [3, N] or None for the
        flow rate (1/L_x) sum u_x.  Returns (dQdF, status, iterations, r)."""
        dQdF = self.torch.empty(3, self.N, dtype=self.torch.float32, device=self.device)
        st, it, r = glbe_adjoint_steady(self.ctx, None if w is None else w.contiguous(), tol, max_iters,
                                        self._adjoint_work(0, 1), dQdF)
        return dQdF, st, it, r

    def adjoint_unrolled(self, nsteps: int, K: int, w=None):
        """Marches nsteps steps (checkpoint every K) and returns dQ/dF [3, N] of
        Q on the final state."""
        dQdF = self.torch.empty(3, self.N, dtype=self.torch.float32, device=self.device)
        glbe_adjoint_unrolled(self.ctx, None if w is None else w.contiguous(), nsteps, K,
                              self._adjoint_work(nsteps, K), dQdF)
        return dQdF


class SteadyVelocity:
    """torch.autograd.Function factory: the steady velocity field as a
    differentiable function of the body-force field.

    ``SteadyVelocity(solver, tol, adj_tol)(F)`` with F [3, N] (FP32, on the
    solver's device) sets the force, solves to r <= tol (glbe_solve from the
    current state) and returns u [3, N].  Its backward takes dL/du as the
    objective weights w and returns dL/dF from the steady adjoint
    (glbe_adjoint_steady) at that state.  The solver must have been created
    with force_field = 3."""

    def __init__(self, solver: "Solver", tol: float = 1e-8, max_steps: int = 10_000_000,
                 adj_tol: float = 1e-6, max_iters: int = 10_000_000):
        import torch
        self.solver, self.tol, self.max_steps = solver, tol, max_steps
        self.adj_tol, self.max_iters = adj_tol, max_iters
        outer = self

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, F):
                S = outer.solver
                S.set_force(F.detach().to(torch.float32).contiguous())
                st, steps, r = S.solve(outer.tol, outer.max_steps)
                if st != GLBE_OK:
                    raise GlbeError(st, "SteadyVelocity forward", f"no steady state (r = {r:g} after {steps})")
                _, u, _ = S.fields()
                return u

            @staticmethod
            def backward(ctx, grad_u):
                S = outer.solver
                dF, st, it, r = S.adjoint_steady(grad_u.detach().to(torch.float32).contiguous(), outer.adj_tol,
                                                 outer.max_iters)
                if st != GLBE_OK:
                    raise GlbeError(st, "SteadyVelocity backward", f"adjoint r = {r:g} after {it} iterations")
                return dF

        self._fn = _Fn

    def __call__(self, F):
        return self._fn.apply(F)
