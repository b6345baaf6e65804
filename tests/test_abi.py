"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads without
a GPU, exports every symbol include/glbe.h declares, and its host-side logic
(defaults, validation, workspace sizing) behaves as documented.  No call here
touches a GPU."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT


def declared_functions(header="glbe.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(glbe(?:2d)?_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0809_4730_gb300 import glbe
    return glbe.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_0809_4730_gb300 import glbe
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in glbe.h but not exported"
        assert n in glbe._SIGNATURES, f"{n} has no Python binding"


def test_library_exports_every_2d_symbol(lib):
    from paper_0809_4730_gb300 import glbe
    names = declared_functions("glbe2d.h")
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), f"{n} declared in glbe2d.h but not exported"
        assert n in glbe._SIGNATURES, f"{n} has no Python binding"


def test_struct_layout_matches(lib):
    from paper_0809_4730_gb300 import glbe
    ps, isz = C.c_size_t(), C.c_size_t()
    lib.glbe_struct_sizes(C.byref(ps), C.byref(isz))
    assert ps.value == C.sizeof(glbe.glbe_params)
    assert isz.value == C.sizeof(glbe.glbe_residual_info)


def test_defaults_are_paper_rates(lib):
    from paper_0809_4730_gb300 import glbe
    p = glbe.glbe_params_default()
    s = list(p.s)
    assert s[1] == 1.19 and s[2] == s[10] == s[12] == 1.4
    assert s[4] == s[6] == s[8] == 1.2 and s[16] == s[17] == s[18] == 1.98
    assert p.rho0 == 1.0 and p.gamma == 1.0 and p.gamma_m == 1.0 and p.storage == glbe.GLBE_F32


def _params(**kw):
    from paper_0809_4730_gb300 import glbe
    p = glbe.glbe_params_default()
    p.nx, p.ny, p.nz = 8, 10, 6
    p.nu = 0.05
    for k, v in kw.items():
        if k in ("wall_lo", "wall_hi", "B0", "F"):
            for d in range(3):
                getattr(p, k)[d] = v[d]
        else:
            setattr(p, k, v)
    return p


def test_workspace_bytes_scales_with_storage_and_induction(lib):
    from paper_0809_4730_gb300 import glbe
    b32 = glbe.glbe_workspace_bytes(_params())
    b16 = glbe.glbe_workspace_bytes(_params(storage=glbe.GLBE_BF16))
    bm = glbe.glbe_workspace_bytes(_params(induction=1, gamma_m=0.5, eta=0.01, chi=0.1))
    N = 8 * 10 * 6
    assert b32 >= 2 * 19 * N * 4
    assert b32 - b16 >= 2 * 19 * N * 2 - 1024
    assert bm - b32 >= 2 * 21 * N * 4 + 3 * N * 4


@pytest.mark.parametrize("bad", [
    dict(gamma=0.0), dict(gamma=1.5), dict(nu=0.0), dict(nx=0),
    dict(wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), ny=2),
    dict(induction=1, gamma_m=0.5, eta=0.0, chi=1.0),
    dict(induction=1, gamma_m=0.5, eta=0.01, chi=0.0),
    dict(force_field=2), dict(storage=7),
])
def test_invalid_parameters_are_rejected(lib, bad):
    from paper_0809_4730_gb300 import glbe
    with pytest.raises(glbe.GlbeError) as ei:
        glbe.glbe_workspace_bytes(_params(**bad))
    assert ei.value.status == glbe.GLBE_ERR_ARG
    assert lib.glbe_last_error()


def test_init_rejects_null_and_small_workspace(lib):
    from paper_0809_4730_gb300 import glbe
    p = _params()
    ctx = C.c_void_p()
    assert lib.glbe_init(C.byref(p), None, 1 << 20, C.byref(ctx)) == glbe.GLBE_ERR_ARG
    assert not ctx.value
    # misaligned pointer is rejected before any CUDA call
    assert lib.glbe_init(C.byref(p), C.c_void_p(0x1001), 1 << 30, C.byref(ctx)) == glbe.GLBE_ERR_ARG
    # too small
    assert lib.glbe_init(C.byref(p), C.c_void_p(0x100000), 16, C.byref(ctx)) == glbe.GLBE_ERR_ARG


def test_null_context_calls_fail_cleanly(lib):
    from paper_0809_4730_gb300 import glbe
    assert lib.glbe_step_n(None, 1) == glbe.GLBE_ERR_ARG
    assert lib.glbe_sync(None) == glbe.GLBE_ERR_ARG
    lib.glbe_destroy(None)


# -- the 2D entry points (include/glbe2d.h) -----------------------------------
def _params2d(**kw):
    from paper_0809_4730_gb300 import glbe
    return glbe.make_params2d(kw.pop("nx", 12), kw.pop("ny", 10), nu=kw.pop("nu", 0.05), **kw)


def test_2d_struct_and_defaults(lib):
    from paper_0809_4730_gb300 import glbe
    p = glbe.glbe2d_params_default()
    assert list(p.s) == [1.0, 1.63, 1.14, 1.0, 1.92, 1.0, 1.92, 1.0, 1.0]
    assert p.rho0 == 1.0 and p.gamma == 1.0 and p.gamma_m == 1.0 and p.storage == glbe.GLBE_F32
    assert p.chi == 1.0 and p.mu == 1.0 and p.induction == 0 and p.force_field == 0


def test_2d_workspace_bytes_scales_with_storage_and_induction(lib):
    from paper_0809_4730_gb300 import glbe
    N = 12 * 10
    b32 = glbe.glbe2d_workspace_bytes(_params2d())
    b16 = glbe.glbe2d_workspace_bytes(_params2d(storage="bf16"))
    bc = glbe.glbe2d_workspace_bytes(_params2d(storage="f32c"))
    bm = glbe.glbe2d_workspace_bytes(_params2d(induction=1, gamma_m=0.5, eta=0.01, chi=0.1))
    bf = glbe.glbe2d_workspace_bytes(_params2d(force_field=2))
    assert b32 >= 2 * 9 * N * 4 + 4 * N * 4
    assert b32 - b16 >= 2 * 9 * N * 2 - 1024
    assert bc - b32 >= 2 * 9 * N * 2 - 1024
    assert bm - b32 >= 2 * 10 * N * 4 + 2 * N * 4
    assert bf - b32 >= 2 * N * 4


@pytest.mark.parametrize("bad", [
    dict(gamma=0.0), dict(gamma=1.5), dict(nu=0.0), dict(nx=0),
    dict(wall_lo=(0, 1), wall_hi=(0, 1), ny=2), dict(wall_lo=(1, 0), wall_hi=(1, 0), nx=2),
    dict(induction=1, gamma_m=0.5, eta=0.0, chi=1.0), dict(induction=1, gamma_m=1.5, eta=0.1),
    dict(induction=1, gamma_m=0.5, eta=0.01, chi=0.0), dict(force_field=1), dict(force_field=3),
    dict(storage=2), dict(storage=4), dict(s=[1.0, 2.0, 1.14, 1.0, 1.92, 1.0, 1.92, 1.0, 1.0]),
])
def test_2d_invalid_parameters_are_rejected(lib, bad):
    from paper_0809_4730_gb300 import glbe
    with pytest.raises(glbe.GlbeError) as ei:
        glbe.glbe2d_workspace_bytes(_params2d(**bad))
    assert ei.value.status == glbe.GLBE_ERR_ARG
    assert lib.glbe_last_error()


def test_2d_init_rejects_null_and_small_workspace_and_null_context(lib):
    from paper_0809_4730_gb300 import glbe
    p = _params2d()
    ctx = C.c_void_p()
    assert lib.glbe2d_init(C.byref(p), None, 1 << 20, C.byref(ctx)) == glbe.GLBE_ERR_ARG
    assert not ctx.value
    assert lib.glbe2d_init(C.byref(p), C.c_void_p(0x1001), 1 << 30, C.byref(ctx)) == glbe.GLBE_ERR_ARG
    assert lib.glbe2d_init(C.byref(p), C.c_void_p(0x100000), 16, C.byref(ctx)) == glbe.GLBE_ERR_ARG
    assert lib.glbe2d_step_n(None, 1) == glbe.GLBE_ERR_ARG
    assert lib.glbe2d_sync(None) == glbe.GLBE_ERR_ARG
    assert lib.glbe2d_set_force(None, None) == glbe.GLBE_ERR_ARG
    lib.glbe2d_destroy(None)


def test_adjoint_workspace_holds_cotangents_and_linearisation_rows(lib):
    """Steady adjoint: two cotangent buffers of 43N floats and the 16N
    linearisation rows of the fixed state (7N without induction); the
    unrolled form adds ceil(nsteps/K) checkpoints and min(K, nsteps)
    recomputed states instead of the rows."""
    from paper_0809_4730_gb300 import glbe
    pm = _params(induction=1, gamma_m=0.5, eta=0.01, chi=0.1)
    pf = _params()
    N = 8 * 10 * 6
    steady_m = glbe.glbe_adjoint_workspace_bytes(pm, 0, 1)
    steady_f = glbe.glbe_adjoint_workspace_bytes(pf, 0, 1)
    assert steady_m >= 2 * 43 * N * 4 + 16 * N * 4
    assert steady_f >= 2 * 43 * N * 4 + 7 * N * 4
    assert steady_m - steady_f >= 9 * N * 4 - 256
    state_m = 19 * N * 4 + 21 * N * 4 + 3 * N * 4
    unrolled = glbe.glbe_adjoint_workspace_bytes(pm, 200, 20)
    assert unrolled >= 2 * 43 * N * 4 + (10 + 20) * state_m
    with pytest.raises(glbe.GlbeError):
        glbe.glbe_adjoint_workspace_bytes(pm, -1, 1)
    with pytest.raises(glbe.GlbeError):
        glbe.glbe_adjoint_workspace_bytes(pm, 10, 0)
